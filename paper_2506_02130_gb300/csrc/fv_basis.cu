// Spectral-basis route (Appendix A): the basis, the per-source coefficient
// kernels, the per-target constants, the interpolation that expands the
// basis at every channel, and the scatter of all channels of a time.
#include "fv_basis.cuh"
#include "fv_plan.cuh"

#include <cmath>
#include <math.h>
#include <vector>

namespace fv {

namespace {

// Exponential-of-semicircle kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on [-1, 1], zero outside
// (Section 2.2, spreading step).
__device__ __forceinline__ double es_phi(double z, double beta)
{
    const double t = 1.0 - z * z;
    return t >= 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}
__device__ __forceinline__ float es_phi(float z, float beta)
{
    const float t = 1.0f - z * z;
    return t >= 0.0f ? expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}

}  // namespace

// ------------------------------------------------------------------ flux coefficients (Eq. A1)
__global__ void __launch_bounds__(256) k_basis_sky(const void *__restrict__ flux, int flux_fp64, long n_src,
                                                   int n_freq, const double *__restrict__ M, int K,
                                                   double *__restrict__ shat)
{
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_src) return;
    double acc[kBasisMax];
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k) acc[k] = 0.0;
    for (int q = 0; q < n_freq; ++q) {
        const size_t idx = (size_t)n * n_freq + q;
        const double I = flux_fp64 ? ((const double *)flux)[idx] : (double)((const float *)flux)[idx];
#pragma unroll
        for (int k = 0; k < kBasisMax; ++k)
            if (k < K) acc[k] += M[q * K + k] * I;
    }
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k)
        if (k < K) shat[(size_t)n * K + k] = acc[k];
}

cudaError_t launch_basis_sky(const void *flux, int flux_fp64, long n_src, int n_freq, const double *M, int K,
                             double *shat, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    if (K < 1 || K > kBasisMax) return cudaErrorInvalidValue;
    k_basis_sky<<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(flux, flux_fp64, n_src, n_freq, M, K, shat);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per time: strengths (Eqs. A2-A3)
// One thread per visible source.  The beam, its coefficients and the product coefficients are computed
// in the grid precision G (the mixed path's strengths are FP32 anyway, and GB300's FP64 rate is a small
// fraction of its FP32 rate); the prephase argument and the grid coordinates in FP64.  The structure
// constants sit in shared memory, read as broadcasts.
template <class G>
__global__ void __launch_bounds__(128) k_prep_basis(const double *__restrict__ sdir, const int *__restrict__ sidx,
                                                    const int *__restrict__ nv_ptr, long n_src,
                                                    const double *__restrict__ shat, const G *__restrict__ M,
                                                    const G *__restrict__ dK, const double *__restrict__ freq,
                                                    int n_freq, int K, int Kp, SliceGeom g, int *__restrict__ cell,
                                                    G *__restrict__ frac, cpx<G> *__restrict__ cs)
{
    __shared__ G s_d[kBasisMax * kBasisMax * kBasisMax];
    const int KKK = K * K * K;
    for (int e = threadIdx.x; e < KKK; e += blockDim.x) s_d[e] = dK[e];
    __syncthreads();
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= *nv_ptr) return;
    const double s0 = sdir[i], s1 = sdir[n_src + i], s2 = sdir[2 * n_src + i];
    const long n = sidx[i];
    const G rho = (G)sqrt(s0 * s0 + s1 * s1), up = (G)s2, east = (G)s0, north = (G)s1;
    // beam coefficients b_hat_k = sum_q M_qk B(nu_q)
    G bh[kBasisMax];
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k) bh[k] = (G)0;
    for (int q = 0; q < n_freq; ++q) {
        const G nu = (G)freq[q];
        const G A = beam_voltage<G>(g.beam, east, north, rho, up, nu, q);
        const G B = g.two_beams ? A * beam_voltage<G>(g.beam2, east, north, rho, up, nu, q) : A * A;
#pragma unroll
        for (int k = 0; k < kBasisMax; ++k)
            if (k < K) bh[k] += M[q * K + k] * B;
    }
    // v_k = sum_i s_hat_i sum_j b_hat_j d^k_ij
    G v[kBasisMax];
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k) v[k] = (G)0;
    for (int a = 0; a < K; ++a) {
        const G sa = (G)shat[(size_t)n * K + a];
        const G *da = s_d + a * K * K;
#pragma unroll
        for (int j = 0; j < kBasisMax; ++j) {
            if (j < K) {
                const G c = sa * bh[j];
#pragma unroll
                for (int k = 0; k < kBasisMax; ++k)
                    if (k < K) v[k] += c * da[j * K + k];
            }
        }
    }
    // prephase e^{i D.(s - C)}: argument and reduction in FP64, sincos in G
    const double st[3] = {s0 - g.dim[0].C, s1 - g.dim[1].C, s2 - g.dim[2].C};
    double ph = 0.0;
    for (int k = 0; k < g.d; ++k) ph += g.dim[k].D * st[k];
    ph -= 6.283185307179586476925 * rint(ph * 0.15915494309189533577);
    G sp, cp;
    if (sizeof(G) == 4) { float a, b; sincosf((float)ph, &a, &b); sp = (G)a; cp = (G)b; }
    else { double a, b; sincos(ph, &a, &b); sp = (G)a; cp = (G)b; }
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k) {
        if (k < K) cs[(size_t)k * n_src + i] = cmk<G>(v[k] * cp, v[k] * sp);
        else if (k < Kp) cs[(size_t)k * n_src + i] = cmk<G>((G)0, (G)0);
    }
    // grid coordinates, split in FP64
    for (int k = 0; k < 3; ++k) {
        if (k < g.d) {
            const double q = st[k] * g.dim[k].qscale;
            const double l0 = ceil(q - 0.5 * g.w);
            cell[(size_t)k * n_src + i] = (int)l0 + g.dim[k].nf1 / 2;
            frac[(size_t)k * n_src + i] = (G)(l0 - q);
        } else {
            cell[(size_t)k * n_src + i] = 0;
            frac[(size_t)k * n_src + i] = (G)0;
        }
    }
}

template <class G>
cudaError_t launch_prep_basis(const double *sdir, const int *sidx, const int *nv_ptr, long n_src, const double *shat,
                              const G *M, const G *dK, const double *freq, int n_freq, int K, int Kp,
                              const SliceGeom &g, int *cell, G *frac, cpx<G> *cs, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    if (K < 1 || K > kBasisMax || Kp < K || Kp > kBasisMax) return cudaErrorInvalidValue;
    k_prep_basis<G><<<(unsigned)((n_src + 127) / 128), 128, 0, st>>>(sdir, sidx, nv_ptr, n_src, shat, M, dK, freq,
                                                                     n_freq, K, Kp, g, cell, frac, cs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per target constants
// The targets (u, q) of a plan and its grid are the same at every time, so each target's footprint
// origin m0 and offsets fr on the FFT grid (Section 2.2 step 3b) and the factor applied after the
// interpolation, the deconvolution prod_i (4/w^2)/Phihat(a_i) times the postphase e^{i x.C}, are
// computed once, in FP64: x = -kappa_q b_u, p = (x - D) M / (2 sigma X), m0 = ceil(p - w/2),
// fr = p - m0, a = (x - D) / X * w pi / (2 sigma), Phihat by the plan's quadrature.
template <class G>
__global__ void k_basis_targets(const double *__restrict__ bu, int n_u, const double *__restrict__ kappa,
                                int n_freq, SliceGeom g, double X0, double X1, double X2, double sigma,
                                const double *__restrict__ gl_x, const double *__restrict__ gl_w, int nq,
                                int4 *__restrict__ tm, G *__restrict__ tf, cpx<G> *__restrict__ ts)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)n_u * n_freq) return;
    const int u = (int)(e / n_freq), q = (int)(e % n_freq);
    const double Xc[3] = {X0, X1, X2};
    const int w = g.w;
    int m0[3] = {0, 0, 0};
    double fr[3] = {0.0, 0.0, 0.0};
    double r = 1.0, ph = 0.0;
    for (int i = 0; i < g.d; ++i) {
        const double x = -kappa[q] * bu[3 * u + i];
        const double p = (x - g.dim[i].D) * g.dim[i].pscale;
        const double m = ceil(p - 0.5 * w);
        m0[i] = (int)m;
        fr[i] = p - m;
        const double a = (x - g.dim[i].D) / Xc[i] * (w * M_PI / (2.0 * sigma));
        double phi_hat = 0.0;
        for (int k = 0; k < nq; ++k) phi_hat += gl_w[k] * es_phi(gl_x[k], g.beta) * cos(a * gl_x[k]);
        r *= (4.0 / ((double)w * w)) / phi_hat;
        ph += x * g.dim[i].C;
    }
    double sp, cp;
    sincos(ph, &sp, &cp);
    tm[e] = make_int4(m0[0], m0[1], m0[2], 0);
#pragma unroll
    for (int i = 0; i < 3; ++i) tf[4 * e + i] = (G)fr[i];
    tf[4 * e + 3] = (G)0;
    ts[e] = cmk<G>((G)(r * cp), (G)(r * sp));
}

template <class G>
cudaError_t launch_basis_targets(const double *bu, int n_u, const double *kappa, int n_freq, const SliceGeom &g,
                                 const double *X, double sigma, const double *gl_x, const double *gl_w, int nq,
                                 int4 *tm, G *tf, cpx<G> *ts, cudaStream_t st)
{
    const long n = (long)n_u * n_freq;
    if (n <= 0) return cudaSuccess;
    k_basis_targets<G><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(bu, n_u, kappa, n_freq, g, X[0], X[1], X[2],
                                                                    sigma, gl_x, gl_w, nq, tm, tf, ts);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ interpolation with the expansion
// One warp per target (u, q).  The band after the x and y passes holds, per (b_y, b_x) cell, the K
// planes' z values contiguously ([k][l_z], K * Nz values).  Lane L holds the values j = L + 32 r
// (r < R = ceil(K Nz / 32)) of that run, with the weights c_j = M_qk K(l_z), where
// K(l_z) = sum_{m_z} phi((2/w)(p_z - m_z)) e^{2 pi i l_z m_z / M_z} (z prescale folded in) is the
// direct z sum of the short z axis; each footprint tap is then R coalesced loads per warp, scaled by
// the tap's x and y kernel values, and the warp reduces at the end.  The target's constants come from
// the per-target table, so the kernel does no FP64 arithmetic.
template <class G, bool HASZ, int R>
__global__ void __launch_bounds__(256) k_interp_basis(const cpx<G> *__restrict__ band, int u0, int n_ug, int n_u,
                                                      int n_freq, const G *__restrict__ M, int K,
                                                      const int *__restrict__ perm, const int4 *__restrict__ tm,
                                                      const G *__restrict__ tf, const cpx<G> *__restrict__ ts,
                                                      G beta, SliceGeom g,
                                                      const G *__restrict__ prez, const cpx<G> *__restrict__ twz,
                                                      cpx<double> *__restrict__ Vq)
{
    const int lane = threadIdx.x & 31;
    const long tg = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    if (tg >= (long)n_ug * n_freq) return;     // whole warps
    // targets in the plan's grid order (perm), so that neighbouring warps read neighbouring footprints
    const int tix_i = perm[(long)u0 * n_freq + tg];
    const size_t tix = (size_t)tix_i;
    const int u = tix_i / n_freq, q = tix_i - u * n_freq;
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w;
    const int4 mm = tm[tix];
    const G frx = tf[4 * tix], fry = tf[4 * tix + 1], frz = tf[4 * tix + 2];
    const int Nz = HASZ ? g.dim[2].nf1 : 1;
    // lane lz < Nz builds K(l_z)
    cpx<G> Kmine = cmk<G>((G)1, (G)0);
    if (HASZ && lane < Nz) {
        const int Mz = g.dim[2].M;
        const int lc = lane - Nz / 2;
        cpx<G> acc = cmk<G>((G)0, (G)0);
        int e = (lc * mm.z) % Mz;
        if (e < 0) e += Mz;
        int step = lc % Mz;
        if (step < 0) step += Mz;
        for (int jz = 0; jz < w; ++jz) {
            const G wt = es_phi(two_over_w * (frz - (G)jz), beta);
            acc = cadd(acc, cscale(twz[e], wt));
            e += step;
            if (e >= Mz) e -= Mz;
        }
        Kmine = cscale(acc, prez[lane]);
    }
    // this lane's weights c_r = M_qk K(l_z) for j = lane + 32 r (shuffles taken by every lane)
    const int KN = K * Nz;                      // R = ceil(KN / 32), a template parameter
    cpx<G> cf[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cf[r] = cmk<G>((G)0, (G)0);
        {
            const int j = lane + 32 * r;
            const bool valid = j < KN;
            const int k = valid ? j / Nz : 0;
            const int lz = valid ? j - k * Nz : 0;
            const G kx = __shfl_sync(0xffffffffu, Kmine.x, lz);
            const G ky = __shfl_sync(0xffffffffu, Kmine.y, lz);
            if (valid) {
                const G mk = M[q * K + k];
                cf[r] = cmk<G>(kx * mk, ky * mk);
            }
        }
    }
    const int Bx = g.dim[0].B;
    const int bx0 = mm.x + g.dim[0].H, by0 = mm.y + g.dim[1].H;
    // x and y kernel values: lane j < w holds the j-th
    const G wxm = lane < w ? es_phi(two_over_w * (frx - (G)lane), beta) : (G)0;
    const G wym = lane < w ? es_phi(two_over_w * (fry - (G)lane), beta) : (G)0;
    G ax = (G)0, ay = (G)0;
    for (int jy = 0; jy < w; ++jy) {
        const G wy = __shfl_sync(0xffffffffu, wym, jy);
        const cpx<G> *row = band + ((size_t)(by0 + jy) * Bx + bx0) * KN;
        for (int jx = 0; jx < w; ++jx) {
            const G wt = wy * __shfl_sync(0xffffffffu, wxm, jx);
            const cpx<G> *c = row + (size_t)jx * KN;
            G sx = (G)0, sy = (G)0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = lane + 32 * r;
                if (r < R - 1 || j < KN) {
                    const cpx<G> v = c[j];
                    sx += v.x * cf[r].x - v.y * cf[r].y;
                    sy += v.x * cf[r].y + v.y * cf[r].x;
                }
            }
            ax += wt * sx;
            ay += wt * sy;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
        const cpx<G> v = cmul(cmk<G>(ax, ay), ts[tix]);
        Vq[(size_t)q * n_u + u] = cmk<double>((double)v.x, (double)v.y);
    }
}

template <class G, bool HASZ, int R>
static void interp_basis_launch(unsigned blocks, const cpx<G> *band, int u0, int n_ug, int n_u, int n_freq,
                                const G *M, int K, const int *perm, const int4 *tm, const G *tf, const cpx<G> *ts,
                                const SliceGeom &g, const G *prez, const cpx<G> *twz, cpx<double> *Vq,
                                cudaStream_t st)
{
    k_interp_basis<G, HASZ, R><<<blocks, 256, 0, st>>>(band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts,
                                                       (G)g.beta, g, prez, twz, Vq);
}

template <class G>
cudaError_t launch_interp_basis(const cpx<G> *band, int u0, int n_ug, int n_u, int n_freq, const G *M, int K,
                                const int *perm, const int4 *tm, const G *tf, const cpx<G> *ts, const SliceGeom &g,
                                const G *prez, const cpx<G> *twz, cpx<double> *Vq, cudaStream_t st)
{
    if (n_ug <= 0) return cudaSuccess;
    const int Nz = g.d == 3 ? g.dim[2].nf1 : 1;
    if (K < 1 || K > kBasisMax || Nz > FV_ZDIRECT_MAX || K * Nz > 256 || g.w > 32) return cudaErrorInvalidValue;
    const long threads = (long)n_ug * n_freq * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const int R = (K * Nz + 31) / 32;
    if (g.d == 3) {
        switch (R) {
        case 1: interp_basis_launch<G, true, 1>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 2: interp_basis_launch<G, true, 2>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 3: interp_basis_launch<G, true, 3>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 4: interp_basis_launch<G, true, 4>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 5: interp_basis_launch<G, true, 5>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 6: interp_basis_launch<G, true, 6>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        case 7: interp_basis_launch<G, true, 7>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        default: interp_basis_launch<G, true, 8>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st); break;
        }
    } else {
        // a flat grid: Nz = 1, K <= 16 values per cell
        interp_basis_launch<G, false, 1>(blocks, band, u0, n_ug, n_u, n_freq, M, K, perm, tm, tf, ts, g, prez, twz, Vq, st);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fit of the spectra (automatic K)
// For source n at time blockIdx.y (rotation R[9 * blockIdx.y]), above the horizon: its spectrum
// c_q = B(nu_q) I_q with the beam pair (b1, b2), the coefficients s_hat = M^T I, b_hat = M^T B and
// c_hat = M^T c over the Kmax columns of M, and for every K <= Kmax the squared distance of the
// route's spectrum M_K v_K (v_K = sum_ij s_hat_i b_hat_j d^k_ij over i, j, k < K) from c, which the
// orthonormal columns give as |v_K|^2 - 2 v_K . c_hat + |c|^2.  Warp sums go to err[K - 1] and
// err[Kmax] (the total |c|^2).  The first K columns of the Kmax basis are the K basis (Gram-Schmidt
// keeps earlier columns), so d_K is the leading block of d_Kmax.
__global__ void __launch_bounds__(128) k_basis_fit(const double *__restrict__ e, long n_src, const double *__restrict__ R,
                                                   const void *__restrict__ flux, int flux_fp64, int n_freq,
                                                   const double *__restrict__ freq, const double *__restrict__ M,
                                                   const double *__restrict__ dK, int Kmax, BeamParams b1,
                                                   BeamParams b2, int two_beams, double *__restrict__ err)
{
    const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const double *Rt = R + 9 * blockIdx.y;
    double sh[kBasisMax], bh[kBasisMax], ch[kBasisMax];
#pragma unroll
    for (int k = 0; k < kBasisMax; ++k) sh[k] = bh[k] = ch[k] = 0.0;
    double cc = 0.0;
    bool up = false;
    if (n < n_src) {
        const double ex = e[n], ey = e[n_src + n], ez = e[2 * n_src + n];
        const double s0 = Rt[0] * ex + Rt[1] * ey + Rt[2] * ez;
        const double s1 = Rt[3] * ex + Rt[4] * ey + Rt[5] * ez;
        const double s2 = Rt[6] * ex + Rt[7] * ey + Rt[8] * ez;
        up = s2 > 0.0;
        if (up) {
            const double rho = sqrt(s0 * s0 + s1 * s1);
            for (int q = 0; q < n_freq; ++q) {
                const double nu = freq[q];
                const double A = beam_voltage<double>(b1, s0, s1, rho, s2, nu, q);
                const double B = two_beams ? A * beam_voltage<double>(b2, s0, s1, rho, s2, nu, q) : A * A;
                const size_t idx = (size_t)n * n_freq + q;
                const double I = flux_fp64 ? ((const double *)flux)[idx] : (double)((const float *)flux)[idx];
                const double c = B * I;
                cc += c * c;
#pragma unroll
                for (int k = 0; k < kBasisMax; ++k)
                    if (k < Kmax) {
                        const double m = M[q * Kmax + k];
                        sh[k] += m * I;
                        bh[k] += m * B;
                        ch[k] += m * c;
                    }
            }
        }
    }
    const int lane = threadIdx.x & 31;
    for (int K = 1; K <= Kmax; ++K) {
        double e2 = 0.0;
        if (up) {
            double v[kBasisMax];
#pragma unroll
            for (int k = 0; k < kBasisMax; ++k) v[k] = 0.0;
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int j = 0; j < kBasisMax; ++j)
                    if (j < K) {
                        const double c = sh[a] * bh[j];
#pragma unroll
                        for (int k = 0; k < kBasisMax; ++k)
                            if (k < K) v[k] += c * dK[((size_t)a * Kmax + j) * Kmax + k];
                    }
            double vv = 0.0, vc = 0.0;
#pragma unroll
            for (int k = 0; k < kBasisMax; ++k)
                if (k < K) {
                    vv += v[k] * v[k];
                    vc += v[k] * ch[k];
                }
            e2 = vv - 2.0 * vc + cc;
        }
        for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
        if (lane == 0) atomicAdd(&err[K - 1], e2);
    }
    for (int o = 16; o > 0; o >>= 1) cc += __shfl_down_sync(0xffffffffu, cc, o);
    if (lane == 0) atomicAdd(&err[Kmax], cc);
}

cudaError_t launch_basis_fit(const double *e, long n_src, const double *R, int n_times, const void *flux,
                             int flux_fp64, int n_freq, const double *freq, const double *M, const double *dK,
                             int Kmax, const BeamParams &b1, const BeamParams &b2, int two_beams, double *err,
                             cudaStream_t st)
{
    if (n_src <= 0 || n_times <= 0) return cudaSuccess;
    if (Kmax < 1 || Kmax > kBasisMax) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((n_src + 127) / 128), (unsigned)n_times);
    k_basis_fit<<<grid, 128, 0, st>>>(e, n_src, R, flux, flux_fp64, n_freq, freq, M, dK, Kmax, b1, b2, two_beams,
                                      err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scatter of all channels of a time
__global__ void k_scatter_basis(const cpx<double> *__restrict__ Vq, const int *__restrict__ bl2u, int n_bl, int n_u,
                                int n_freq, int n_time, int t, char *__restrict__ vis, size_t slice_bytes,
                                int out_fp64)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)n_bl * n_freq) return;
    const int q = (int)(e / n_bl), bl = (int)(e % n_bl);
    const cpx<double> v = Vq[(size_t)q * n_u + bl2u[bl]];
    char *slice = vis + ((size_t)q * n_time + t) * slice_bytes;
    if (out_fp64)
        reinterpret_cast<double2 *>(slice)[bl] = make_double2(v.x, v.y);
    else
        reinterpret_cast<float2 *>(slice)[bl] = make_float2((float)v.x, (float)v.y);
}

cudaError_t launch_scatter_basis(const cpx<double> *Vq, const int *bl2u, int n_bl, int n_u, int n_freq, int n_time,
                                 int t, char *vis, size_t slice_bytes, int out_fp64, cudaStream_t st)
{
    const long n = (long)n_bl * n_freq;
    if (n <= 0) return cudaSuccess;
    k_scatter_basis<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Vq, bl2u, n_bl, n_u, n_freq, n_time, t, vis,
                                                                 slice_bytes, out_fp64);
    return cudaGetLastError();
}

template cudaError_t launch_prep_basis<float>(const double *, const int *, const int *, long, const double *,
                                              const float *, const float *, const double *, int, int, int,
                                              const SliceGeom &, int *, float *, cpx<float> *, cudaStream_t);
template cudaError_t launch_prep_basis<double>(const double *, const int *, const int *, long, const double *,
                                               const double *, const double *, const double *, int, int, int,
                                               const SliceGeom &, int *, double *, cpx<double> *, cudaStream_t);
template cudaError_t launch_interp_basis<float>(const cpx<float> *, int, int, int, int, const float *, int,
                                                const int *, const int4 *, const float *, const cpx<float> *,
                                                const SliceGeom &, const float *, const cpx<float> *, cpx<double> *,
                                                cudaStream_t);
template cudaError_t launch_interp_basis<double>(const cpx<double> *, int, int, int, int, const double *, int,
                                                 const int *, const int4 *, const double *, const cpx<double> *,
                                                 const SliceGeom &, const double *, const cpx<double> *,
                                                 cpx<double> *, cudaStream_t);
template cudaError_t launch_basis_targets<float>(const double *, int, const double *, int, const SliceGeom &,
                                                 const double *, double, const double *, const double *, int, int4 *,
                                                 float *, cpx<float> *, cudaStream_t);
template cudaError_t launch_basis_targets<double>(const double *, int, const double *, int, const SliceGeom &,
                                                  const double *, double, const double *, const double *, int,
                                                  int4 *, double *, cpx<double> *, cudaStream_t);

}  // namespace fv

// ------------------------------------------------------------------ the basis (host)
// Chebyshev polynomials T_0..T_{K-1} of x = (2 nu - nu_min - nu_max) / (nu_max - nu_min) at the
// channels, orthonormalised column by column with modified Gram-Schmidt, each column twice (the
// second sweep removes what rounding left of the earlier directions).  Fails if a column has no
// component left (fewer distinct channels than K).
bool basis_matrix(const std::vector<double> &freq, int K, std::vector<double> &M)
{
    const int nq = (int)freq.size();
    if (K < 1 || K > nq) return false;
    double lo = freq[0], hi = freq[0];
    for (double f : freq) { lo = std::min(lo, f); hi = std::max(hi, f); }
    M.assign((size_t)nq * K, 0.0);
    for (int q = 0; q < nq; ++q) {
        const double x = hi > lo ? (2.0 * freq[q] - lo - hi) / (hi - lo) : 0.0;
        double t0 = 1.0, t1 = x;
        for (int k = 0; k < K; ++k) {
            double tk;
            if (k == 0) tk = t0;
            else if (k == 1) tk = t1;
            else { tk = 2.0 * x * t1 - t0; t0 = t1; t1 = tk; }
            M[(size_t)q * K + k] = tk;
        }
    }
    for (int k = 0; k < K; ++k) {
        double n0 = 0.0;
        for (int q = 0; q < nq; ++q) n0 += M[(size_t)q * K + k] * M[(size_t)q * K + k];
        for (int sweep = 0; sweep < 2; ++sweep)
            for (int j = 0; j < k; ++j) {
                double dot = 0.0;
                for (int q = 0; q < nq; ++q) dot += M[(size_t)q * K + j] * M[(size_t)q * K + k];
                for (int q = 0; q < nq; ++q) M[(size_t)q * K + k] -= dot * M[(size_t)q * K + j];
            }
        double nn = 0.0;
        for (int q = 0; q < nq; ++q) nn += M[(size_t)q * K + k] * M[(size_t)q * K + k];
        if (!(nn > 1e-24 * n0) || !(nn > 0.0)) return false;
        const double inv = 1.0 / std::sqrt(nn);
        for (int q = 0; q < nq; ++q) M[(size_t)q * K + k] *= inv;
    }
    return true;
}
