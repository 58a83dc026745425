// Internal declarations shared by the translation units of libfftvis_gb300.
//
// Notation (Section 2.2, Eq. 4-5): sources s_n are topocentric direction
// cosines (E, N, U); targets x_k = -2 pi nu b_k / c; the result of one slice is
// f_k = sum_n c_n exp(i x_k . s_n).  The type-3 transform is evaluated as
//   f_k = e^{i x_k.C} * prod_i (4/w^2)/Phihat(a_ki)
//         * sum_m prod_i phi((2/w)(p_ki - m_i)) * P_m,
//   P_m = sum_l g_l prod_i [1/Phihat(l_i w pi / M_i)] e^{2 pi i l.m/M},
//   g_l = sum_n c_n e^{i D.(s_n - C)} prod_i phi((2/w)(l_i - q_ni)),
// with C, S the centre and half-extent of the sources, D, X those of the
// targets, q = (s - C) sigma X / pi the source grid coordinate (cells),
// p = (x - D) M / (2 sigma X) the target coordinate on the FFT grid of M
// points, a = (x - D) w pi / (2 sigma X), phi the ES kernel of Section 2.2
// (step 1) and Phihat(k) = int_{-1}^{1} phi(z) cos(k z) dz.  The grid size
// per dimension is nf1 >= 2 sigma X S / pi + w (Eq. 5).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FV_C_LIGHT 299792458.0
#define FV_MAX_STAGES 8
#define FV_ZDIRECT_MAX 16

namespace fv {

template <class T> struct cpx { T x, y; };

template <class T> __host__ __device__ __forceinline__ cpx<T> cmk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <class T> __host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T> __host__ __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return cmk<T>(a.x * s, a.y * s); }
// multiply by +i
template <class T> __host__ __device__ __forceinline__ cpx<T> cmuli(cpx<T> a) { return cmk<T>(-a.y, a.x); }

// Geometry of one dimension of one slice's transform.
struct DimGeom {
    int nf1;        // spreading grid points
    int M;          // FFT length (sigma * nf1, 2^a 3^b 5^c)
    int B;          // band of FFT outputs kept: indices m in [-H, B-1-H]
    int H;          // band offset
    double qscale;  // sigma X / pi : (s - C) -> source grid coordinate (cells)
    double pscale;  // M / (2 sigma X) : (x - D) -> target coordinate (FFT cells)
    double D;       // target centre (rad)
    double C;       // source centre
    int nstages;
    int radix[FV_MAX_STAGES];
    unsigned mr_mul[FV_MAX_STAGES], mr_sh[FV_MAX_STAGES];   // division by M / radix[s]
    unsigned ns_mul[FV_MAX_STAGES], ns_sh[FV_MAX_STAGES];   // division by prod(radix[0..s-1])
};

struct BeamParams {
    int kind;           // 0 gauss, 1 airy, 2 uniform
    double p0, p1, p2;
};

// Per-time binning geometry: bins are tiles of the top (highest-frequency)
// channel's grid in (x, y).
struct TimeBin {
    double R[9];            // equatorial -> ENU rotation at this time
    double C[3];            // source centre
    double qscale_top[3];   // grid scale of the top channel
    int nf1_top[3];
    int T[2];               // tile (= bin) size in cells
    int nbx, nby;           // bins per axis
};

#define FV_SPREAD_SMEM_MAX (96 * 1024)

// Everything a slice's kernels need, passed by value.
struct SliceGeom {
    double R[9];        // equatorial -> ENU rotation at this time (row major)
    double nu;          // Hz
    double kappa;       // 2 pi nu / c
    int d;              // 2 or 3
    int w;              // kernel width
    double beta;        // ES shape
    int n_pol;          // 1 or 4
    int polarized;
    int n_stokes;
    BeamParams beam;
    DimGeom dim[3];
};

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the launch error (cudaSuccess if fine).

// e[3][n]: equatorial unit vectors from (ra, dec).
cudaError_t launch_radec_to_unit(const double *ra, const double *dec, long n, double *e, cudaStream_t st);

// Per-block min/max of visible ENU directions over all times: out[nblocks][6].
cudaError_t launch_source_extents(const double *e, long n, const double *R_all, int n_time,
                                  double *out, int nblocks, cudaStream_t st);

// tab[j] = 1 / Phihat(k_j), k_j = (j - n/2) * w * pi / M  (prescale table of one dim).
template <class G>
cudaError_t launch_prescale_table(G *tab, int nf1, int M, int w, double beta, const double *gl_x,
                                  const double *gl_w, int nq, cudaStream_t st);

// tw[k] = e^{2 pi i k / M}
template <class G>
cudaError_t launch_twiddles(cpx<G> *tw, int M, cudaStream_t st);

// dec[u] = prod_i (4/w^2) / Phihat(a_ui), a = (b_c - b) / b_half * w pi / (2 sigma)
// (channel-independent, Section 2.2 deconvolution), FP64.
cudaError_t launch_target_deconv(const double *bu, int n_u, int d, const double *bcen, const double *bhalf,
                                 int w, double beta, double sigma, const double *gl_x, const double *gl_w,
                                 int nq, double *dec, cudaStream_t st);

// Fused weighting (beam x flux, Eq. 1-3), rotation, horizon cut, prephase and
// spreading with global atomics onto grid [n_pol][nz][ny][nx].
template <class G>
cudaError_t launch_spread_direct(const double *e, long n_src, const void *flux, int flux_fp64, int n_freq,
                                 int f, const SliceGeom &g, cpx<G> *grid, cudaStream_t st);

// Per time: rotate, horizon cut and counting sort of the visible sources by
// top-channel tile.  sdir[3][n_src] and sidx[n_src] hold the sorted visible
// directions and source indices; offsets[nb] is the visible count.
cudaError_t launch_time_binning(const double *e, long n_src, const TimeBin &tb, int *bin_of, int *counts,
                                int *offsets, int *cursor, double *sdir, int *sidx, cudaStream_t st);

// Per slice: strengths with prephase and split grid coordinates of the sorted sources.
template <class G>
cudaError_t launch_prep(const double *sdir, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                        int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, G *frac, cpx<G> *cs,
                        cudaStream_t st);

// Gather-spreading configuration for a grid precision, product count and z
// size: returns 0 if unsupported, else the z template size and the bin size
// (top-channel cells per bin in x and y).
int spread_gather_config(int elem_bytes, int n_pol, int nz, int w, int *nz_tmpl, int *bin_x, int *bin_y);

// Per slice: tiled spreading; writes every cell of grid [n_pol][nz][ny][nx].
template <class G>
cudaError_t launch_spread_tile(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                               const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                               cudaStream_t st);

// Scatter variant of the tiled spreading (shared-memory tile + atomics);
// same inputs and output as launch_spread_tile.
template <class G>
cudaError_t launch_spread_scatter(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                  const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                                  cudaStream_t st);
size_t spread_scatter_smem(int elem_bytes, int n_pol, int nz);

// One FFT pass: rows of length N (input rows contiguous), prescale by pre[l],
// zero-pad to M, FFT with e^{+2 pi i l m / M}, write band outputs transposed:
// out[b][row] = P[(b - H) mod M].
template <class G>
cudaError_t launch_fft_pass(const cpx<G> *in, cpx<G> *out, long rows, const DimGeom &dg, const G *pre,
                            const cpx<G> *tw, cudaStream_t st);

// Interpolation at the unique targets, deconvolution and postphase: Vu[u][pol] (FP64).
template <class G>
cudaError_t launch_interp(const cpx<G> *band, const double *bu, int n_u, const double *dec, const SliceGeom &g,
                          cpx<double> *Vu, cudaStream_t st);

// Same, reading the band after the x and y passes only ([b_y][b_x][pol][l_z]),
// with the z axis summed directly (nf1_z <= 16).
template <class G>
cudaError_t launch_interp_zdirect(const cpx<G> *band, const double *bu, int n_u, const double *dec,
                                  const SliceGeom &g, const G *prez, const cpx<G> *twz, cpx<double> *Vu,
                                  cudaStream_t st);

// vis slice [n_bl][n_pol] (complex128 or complex64) <- Vu[bl2u[bl]].
cudaError_t launch_scatter(const cpx<double> *Vu, const int *bl2u, int n_bl, int n_pol, void *out,
                           int out_fp64, cudaStream_t st);

size_t fft_pass_smem_bytes(int M, int elem_bytes);
int fft_max_M(int elem_bytes);
int fft_rows_per_cta(int M, int elem_bytes);
// Smallest even M >= target that is a product of at most 3 (4 above 4096)
// supported radices; fills radix[] and nstages.  -1 if none.
int fft_choose_length(int target, int *radix, int &nstages, int maxRadix);
// Per-stage multiply-high division constants of dg (needs M, nstages, radix).
void fft_stage_constants(DimGeom &dg);

}  // namespace fv
