// Spectral-basis route (Appendix A): declarations shared by the runtime and
// the route's kernels.
//
// The channels q of a time share one type-3 transform per basis function k:
//   strengths  v_nk = sum_ij s_hat_ni b_hat_nj d^k_ij            (Eqs. A1-A4)
//   transform  T_k(x) = sum_n v_nk e^{i x . s_n}, x = -2 pi nu_q b / c
//   expansion  V(b, nu_q) = sum_k M_qk T_k(x_qb)
// with one grid per time sized for the targets of every channel (Eq. A5).
// The interpolation applies the expansion: each target reads the K planes of
// its footprint and weights plane k by M_qk.
#pragma once
#include "fv_internal.cuh"

namespace fv {

constexpr int kBasisMax = 16;

// s_hat[n][k] = sum_q M[q][k] I_n(nu_q): the flux coefficients of every source (Eq. A1 with
// orthonormal columns, so that (M^T M)^{-1} = 1).  flux: [n_src][n_freq] (Stokes I).
cudaError_t launch_basis_sky(const void *flux, int flux_fp64, long n_src, int n_freq, const double *M, int K,
                             double *shat, cudaStream_t st);

// Per visible source i < *nv_ptr (sorted order of the time binning): beam coefficients
// b_hat = M^T B(nu_.) at its direction with the slice geometry's beams (Eq. A2), product coefficients
// v_k = sum_ij s_hat_i b_hat_j d^k_ij (Eq. A3), both in G; prephase e^{i D.(s - C)} and grid
// coordinates.  M and dK are G copies of the basis and structure constants.  cs: [Kp][n_src], planes
// K..Kp-1 zero.
template <class G>
cudaError_t launch_prep_basis(const double *sdir, const int *sidx, const int *nv_ptr, long n_src, const double *shat,
                              const G *M, const G *dK, const double *freq, int n_freq, int K, int Kp,
                              const SliceGeom &g, int *cell, G *frac, cpx<G> *cs, cudaStream_t st);

// Constants of every target t = u * n_freq + q of the one grid g (target centre D = g.dim[i].D,
// half-extent X[i]): tm[t] = footprint origin (m0_x, m0_y, m0_z, 0) on the FFT grid, tf[4t + i] = offset
// p_i - m0_i, ts[t] = prod_i (4/w^2)/Phihat(a_i) e^{i x.C} with x = -kappa_q b_u,
// a_i = (x_i - D_i) / X_i * w pi / (2 sigma).
template <class G>
cudaError_t launch_basis_targets(const double *bu, int n_u, const double *kappa, int n_freq, const SliceGeom &g,
                                 const double *X, double sigma, const double *gl_x, const double *gl_w, int nq,
                                 int4 *tm, G *tf, cpx<G> *ts, cudaStream_t st);

// Targets (u, q) for u in [u0, u0 + n_ug) and every channel q, taken in the order
// perm[u0 * n_freq .. (u0 + n_ug) * n_freq) (a permutation of that range): interpolation of the K planes
// of the band ([b_y][b_x][k][l_z] after the x and y passes) with the z sum done directly (short z),
// combined with weights M_qk, times the target's constant ts.  Vq[q * n_u + u] receives the result.
template <class G>
cudaError_t launch_interp_basis(const cpx<G> *band, int u0, int n_ug, int n_u, int n_freq, const G *M, int K,
                                const int *perm, const int4 *tm, const G *tf, const cpx<G> *ts, const SliceGeom &g,
                                const G *prez, const cpx<G> *twz, cpx<double> *Vq, cudaStream_t st);

// Spectral fit for the automatic choice of K: over the sources above the horizon at each of the
// n_times rotations R[n_times][9], err[K - 1] += |M_K v_K - B I|^2 (the route's spectrum against the
// exact one, all channels) for K = 1..Kmax and err[Kmax] += |B I|^2, with the beam pair (b1, b2).
// M: [n_freq][Kmax] orthonormal columns, dK: [Kmax]^3.  err must start at zero.
cudaError_t launch_basis_fit(const double *e, long n_src, const double *R, int n_times, const void *flux,
                             int flux_fp64, int n_freq, const double *freq, const double *M, const double *dK,
                             int Kmax, const BeamParams &b1, const BeamParams &b2, int two_beams, double *err,
                             cudaStream_t st);

// Output slices (q, t) of every channel: vis + (q * n_time + t) * slice_bytes holds, for baseline bl,
// Vq[q * n_u + bl2u[bl]] (complex64 or complex128).
cudaError_t launch_scatter_basis(const cpx<double> *Vq, const int *bl2u, int n_bl, int n_u, int n_freq, int n_time,
                                 int t, char *vis, size_t slice_bytes, int out_fp64, cudaStream_t st);

}  // namespace fv
