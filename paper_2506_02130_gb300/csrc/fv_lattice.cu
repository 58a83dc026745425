// Lattice arrays: the type-1 route of Section 2.2.1.
//
// When the antennas of a coplanar array sit on a lattice,
// x_a = x_0 + k_a1 a_1 + k_a2 a_2 with integer k, every baseline is
// b = n_1 a_1 + n_2 a_2 (n = k_i - k_j), and the fringe phase of a source
// becomes -2 pi nu b.s / c = -n . x_s with x_sd = (2 pi nu / c) a_d . s.  A
// slice is then V(n) = sum_s c_s exp(-i n . x_s): a type-1 transform from the
// non-uniform x_s (taken mod 2 pi) to the integer modes |n_d| <= H_d.  This is
// the paper's L b_phys mapping written with the lattice basis (L^{-1} =
// [a_1 a_2]); the sources are mapped by the transpose, s' = L^{-T} s.
//
// Per slice: strengths, the grid coordinate t_d = frac(x_d / 2 pi) nf_d split
// into a first footprint cell and an offset (FP64); spreading with the ES
// kernel onto a periodic nf_x x nf_y grid (a CTA sums a block of sources into
// its own copy of the grid in shared memory, then adds the copy to the grid);
// the two FFT passes of the type-3 path with no zero padding, keeping the
// band of modes m in [-H, H]; and per baseline V(n) = G(-n) / (Psihat_x(n_x)
// Psihat_y(n_y)) with Psihat(n) = (w/2) Phihat(pi w n / nf).
#include "fv_internal.cuh"

#include <math.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

namespace fv {

// ------------------------------------------------------------------ host: lattice detection
int lattice_detect(int n_ant, const double *enu, double tol, double basis[4], int *index)
{
    if (n_ant < 1 || !enu) return 0;
    if (!(tol > 0.0)) tol = 1e-10;
    bool flat = true;
    for (int a = 0; a < n_ant; ++a)
        if (std::fabs(enu[3 * a + 2] - enu[2]) > tol) flat = false;     // heights differ
    std::vector<double> rx(n_ant), ry(n_ant);
    for (int a = 0; a < n_ant; ++a) {
        rx[a] = enu[3 * a] - enu[0];
        ry[a] = enu[3 * a + 1] - enu[1];
    }
    // shortest difference vector, then the shortest one off its line
    const double inf = std::numeric_limits<double>::infinity();
    double b1 = inf, v1x = 0, v1y = 0;
    for (int a = 0; a < n_ant; ++a)
        for (int b = a + 1; b < n_ant; ++b) {
            const double dx = rx[b] - rx[a], dy = ry[b] - ry[a], l2 = dx * dx + dy * dy;
            if (l2 > 100.0 * tol * tol && l2 < b1) { b1 = l2; v1x = dx; v1y = dy; }
        }
    if (b1 == inf) {   // every antenna above one point: all horizontal offsets are zero
        basis[0] = 1.0; basis[1] = 0.0; basis[2] = 0.0; basis[3] = 1.0;
        for (int a = 0; a < 2 * n_ant; ++a) index[a] = 0;
        return flat ? 1 : 2;
    }
    const double l1 = std::sqrt(b1);
    double b2 = inf, v2x = 0, v2y = 0;
    for (int a = 0; a < n_ant; ++a)
        for (int b = a + 1; b < n_ant; ++b) {
            const double dx = rx[b] - rx[a], dy = ry[b] - ry[a], l2 = dx * dx + dy * dy;
            const double off = std::fabs(v1x * dy - v1y * dx) / l1;   // distance from the line of v1
            if (off > 10.0 * tol && l2 < b2) { b2 = l2; v2x = dx; v2y = dy; }
        }
    if (b2 == inf) { v2x = -v1y; v2y = v1x; }   // collinear array: any second vector, all k_2 = 0
    // Lagrange-Gauss reduction of (v1, v2)
    for (int it = 0; it < 64; ++it) {
        const double n1 = v1x * v1x + v1y * v1y, n2 = v2x * v2x + v2y * v2y;
        if (n2 < n1) { std::swap(v1x, v2x); std::swap(v1y, v2y); continue; }
        const double mu = std::nearbyint((v1x * v2x + v1y * v2y) / n1);
        if (mu == 0.0) break;
        v2x -= mu * v1x;
        v2y -= mu * v1y;
    }
    const double det = v1x * v2y - v1y * v2x;
    if (!(std::fabs(det) > 0.0)) return 0;
    for (int a = 0; a < n_ant; ++a) {
        const double k1 = (rx[a] * v2y - ry[a] * v2x) / det, k2 = (v1x * ry[a] - v1y * rx[a]) / det;
        const double r1 = std::nearbyint(k1), r2 = std::nearbyint(k2);
        if (std::fabs(r1) > 1e6 || std::fabs(r2) > 1e6) return 0;
        const double ex = rx[a] - (r1 * v1x + r2 * v2x), ey = ry[a] - (r1 * v1y + r2 * v2y);
        if (std::sqrt(ex * ex + ey * ey) > tol) return 0;
        index[2 * a] = (int)r1;
        index[2 * a + 1] = (int)r2;
    }
    basis[0] = v1x; basis[1] = v1y; basis[2] = v2x; basis[3] = v2y;
    return flat ? 1 : 2;
}

// ------------------------------------------------------------------ device
__device__ __forceinline__ double lat_es_d(double z, double beta)
{
    const double t = 1.0 - z * z;
    return t >= 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}
__device__ __forceinline__ float lat_es_f(float z, float beta)
{
    const float t = 1.0f - z * z;
    return t >= 0.0f ? __expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}
template <class G> __device__ __forceinline__ G lat_es(G z, G beta);
template <> __device__ __forceinline__ double lat_es<double>(double z, double beta) { return lat_es_d(z, beta); }
template <> __device__ __forceinline__ float lat_es<float>(float z, float beta) { return lat_es_f(z, beta); }

template <class G>
__global__ void __launch_bounds__(256) k_prep_lattice(const double *__restrict__ sdir, const int *__restrict__ sidx,
                                                      const int *__restrict__ nv_ptr, long n_src,
                                                      const void *__restrict__ flux, int flux_fp64, int n_freq,
                                                      int f, SliceGeom g, LatGeom lg, int *__restrict__ cell,
                                                      G *__restrict__ frac, cpx<G> *__restrict__ cs)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= *nv_ptr) return;
    const double s0 = sdir[i], s1 = sdir[n_src + i], s2 = sdir[2 * n_src + i];
    const long n = sidx[i];
    cpx<G> c[4];
    const int np = source_strengths<G>(g, s0, s1, s2, n, flux, flux_fp64, n_src, n_freq, f, c);
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (p < np) cs[(size_t)p * n_src + i] = c[p];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const double x = g.kappa * (lg.a[d][0] * s0 + lg.a[d][1] * s1);
        double t = x * 0.15915494309189533577;          // x / 2 pi
        t -= rint(t);                                    // periodic: t in [-1/2, 1/2]
        const double gp = t * lg.nf[d];
        const double l0 = ceil(gp - 0.5 * g.w);
        cell[(size_t)d * n_src + i] = (int)l0 + lg.nf[d] / 2;
        frac[(size_t)d * n_src + i] = (G)(l0 - gp);
    }
    frac[2 * (size_t)n_src + i] = (G)(2.0 * s2 - 1.0);   // Chebyshev argument of the height factor
    // kernel values of the x and y footprints, once per source: kw[i][0..w) (x), kw[i][w..2w) (y)
    G *kw = frac + 3 * (size_t)n_src + (size_t)i * 2 * g.w;
    const G two_over_w = (G)2 / (G)g.w, beta = geom_beta<G>(g);
    const G fx = frac[i], fy = frac[(size_t)n_src + i];
    for (int j = 0; j < g.w; ++j) {
        kw[j] = lat_es<G>(two_over_w * (fx + (G)j), beta);
        kw[g.w + j] = lat_es<G>(two_over_w * (fy + (G)j), beta);
    }
}

template <class G>
cudaError_t launch_prep_lattice(const double *sdir, const int *sidx, const int *nv_ptr, long n_src,
                                const void *flux, int flux_fp64, int n_freq, int f, const SliceGeom &g,
                                const LatGeom &lg, int *cell, G *frac, cpx<G> *cs, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    k_prep_lattice<G><<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(sdir, sidx, nv_ptr, n_src, flux, flux_fp64,
                                                                       n_freq, f, g, lg, cell, frac, cs);
    return cudaGetLastError();
}

// One warp per source: lanes j < w hold the x and y kernel values, the warp
// covers the w x w footprint in rounds of 32 cells (same trip count on every
// lane: shuffles inside) and adds into the grid copies, wrapping periodically;
// the copy of term q receives c T_q(u) (T_q by its three-term recurrence).
// blockIdx.y is the product, blockIdx.z the block of terms [q0, q1).
// SMEM: the copies are in shared memory (split real/imaginary planes) and are
// added to the global grids at the end; otherwise the adds go straight to the
// global grids.
constexpr int kLatMaxTermsPerCta = 8;

constexpr int kLatSpreadThreads = 512;

template <class G, bool SMEM>
__global__ void __launch_bounds__(kLatSpreadThreads) k_spread_lattice(const int *__restrict__ nv_ptr, const int *__restrict__ cell,
                                                        const G *__restrict__ frac, const cpx<G> *__restrict__ cs,
                                                        long n_src, int w, G beta, int nfx, int nfy, int np, int K,
                                                        int kc, long per, cpx<G> *__restrict__ grid)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long nv = *nv_ptr;
    const long start = (long)blockIdx.x * per;
    if (start >= nv) return;                       // the same on every thread of the CTA
    const long end = min(nv, start + per);
    const int p = blockIdx.y;
    const int q0 = blockIdx.z * kc, q1 = min(K, q0 + kc), nq = q1 - q0;   // nq <= kLatMaxTermsPerCta
    const int ncell = nfx * nfy;
    G *sre = reinterpret_cast<G *>(smem_raw);      // [nq][ncell]
    G *sim = sre + (size_t)nq * ncell;
    if (SMEM) {
        for (int idx = threadIdx.x; idx < nq * ncell; idx += blockDim.x) {
            sre[idx] = (G)0;
            sim[idx] = (G)0;
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ww = w * w;
    // this lane's footprint cells in the first two rounds (w <= 8 needs no more)
    const int jy0 = lane / w, jx0 = lane - jy0 * w;
    const int l1 = lane + 32, jy1 = l1 / w, jx1 = l1 - jy1 * w;
    for (long i = start + warp; i < end; i += nwarps) {     // the same trip count on every lane of a warp
        const int cx = cell[i], cy = cell[n_src + i];
        const G u = frac[2 * n_src + i];
        const cpx<G> c = cs[(size_t)p * n_src + i];
        const G *kw = frac + 3 * (size_t)n_src + (size_t)i * 2 * w;   // kernel values from the preparation
        const G wxm = lane < w ? kw[lane] : (G)0;
        const G wym = lane < w ? kw[w + lane] : (G)0;
        // T_q(u) for this CTA's terms, by the three-term recurrence
        G tq[kLatMaxTermsPerCta];
        {
            G tm1 = (G)1, t = (G)1;
            for (int q = 0; q < q0; ++q) {
                const G tn = q == 0 ? u : (G)2 * u * t - tm1;
                tm1 = t;
                t = tn;
            }
#pragma unroll
            for (int j = 0; j < kLatMaxTermsPerCta; ++j) {
                tq[j] = t;
                const G tn = (q0 + j) == 0 ? u : (G)2 * u * t - tm1;
                tm1 = t;
                t = tn;
            }
        }
        for (int base = 0; base < ww; base += 32) {
            const int idx = base + lane;
            const bool valid = idx < ww;
            int jy, jx;
            if (base == 0) { jy = jy0; jx = jx0; }
            else if (base == 32) { jy = jy1; jx = jx1; }
            else { jy = idx / w; jx = idx - jy * w; }
            if (!valid) { jy = 0; jx = 0; }
            const G wt = __shfl_sync(0xffffffffu, wym, jy) * __shfl_sync(0xffffffffu, wxm, jx);
            if (valid) {
                int lx = cx + jx, ly = cy + jy;
                if (lx < 0) lx += nfx; else if (lx >= nfx) lx -= nfx;
                if (ly < 0) ly += nfy; else if (ly >= nfy) ly -= nfy;
                const int o = ly * nfx + lx;
                const cpx<G> cw = cscale(c, wt);
#pragma unroll
                for (int j = 0; j < kLatMaxTermsPerCta; ++j) {
                    if (j < nq) {
                        if (SMEM) {
                            atomicAdd(&sre[(size_t)j * ncell + o], cw.x * tq[j]);
                            atomicAdd(&sim[(size_t)j * ncell + o], cw.y * tq[j]);
                        } else {
                            cpx<G> *gq = grid + ((size_t)(q0 + j) * np + p) * ncell;
                            atomicAdd(&gq[o].x, cw.x * tq[j]);
                            atomicAdd(&gq[o].y, cw.y * tq[j]);
                        }
                    }
                }
            }
        }
    }
    if (SMEM) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < nq * ncell; idx += blockDim.x) {
            const G vr = sre[idx], vi = sim[idx];
            if (vr != (G)0 || vi != (G)0) {
                const int j = idx / ncell, o = idx - j * ncell;
                cpx<G> *gq = grid + ((size_t)(q0 + j) * np + p) * ncell;
                atomicAdd(&gq[o].x, vr);
                atomicAdd(&gq[o].y, vi);
            }
        }
    }
}

static constexpr size_t kLatSmemMax = 200 * 1024;

template <class G>
cudaError_t launch_spread_lattice(const int *nv_ptr, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                  const SliceGeom &g, const LatGeom &lg, cpx<G> *grid, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    static int sms[64] = {};
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev]) {
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    // Terms per CTA: as many as keep the CTA's copy within 96 KB (so that two CTAs share an SM; every
    // term block of a source repeats its kernel values and footprint), at least one if one term fits.  Source blocks: about four CTAs per SM in total,
    // each of at least 512 sources (every CTA adds its whole copy to the grid at the end).
    const size_t plane = 2 * (size_t)lg.nf[0] * lg.nf[1] * sizeof(G);
    int kc = (int)std::min<size_t>((size_t)std::min(lg.K, kLatMaxTermsPerCta), std::max<size_t>(96 * 1024 / plane, 1));
    const bool smem_ok = plane * kc <= kLatSmemMax;
    const int kcu = smem_ok ? kc : std::min(lg.K, kLatMaxTermsPerCta);
    const int nz = (lg.K + kcu - 1) / kcu;
    const long slots = std::max(1L, 4L * sms[dev] / ((long)nz * g.n_pol));
    long nblk = std::max<long>(1, std::min<long>((n_src + 511) / 512, slots));
    const long per = (n_src + nblk - 1) / nblk;
    nblk = (n_src + per - 1) / per;
    dim3 grid_dim((unsigned)nblk, (unsigned)g.n_pol, (unsigned)nz);
    if (smem_ok) {
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(k_spread_lattice<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLatSmemMax);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
        k_spread_lattice<G, true><<<grid_dim, kLatSpreadThreads, plane * kcu, st>>>(nv_ptr, cell, frac, cs, n_src, g.w,
                                                                      (G)g.beta, lg.nf[0], lg.nf[1], g.n_pol, lg.K,
                                                                      kcu, per, grid);
    } else {
        k_spread_lattice<G, false><<<grid_dim, kLatSpreadThreads, 0, st>>>(nv_ptr, cell, frac, cs, n_src, g.w, (G)g.beta,
                                                              lg.nf[0], lg.nf[1], g.n_pol, lg.K, kcu, per, grid);
    }
    return cudaGetLastError();
}

template <class G>
__global__ void k_gather_lattice(const cpx<G> *__restrict__ band, const int *__restrict__ bln,
                                 const int *__restrict__ bl_list, int n_bl, int n_pol, LatGeom lg,
                                 const cpx<double> *__restrict__ wq, const double *__restrict__ dx,
                                 const double *__restrict__ dy, void *out, int out_fp64)
{
    const long j = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (j >= (long)n_bl * n_pol) return;
    const long jb = j / n_pol;
    const int p = (int)(j - jb * n_pol);
    const long b = bl_list ? bl_list[jb] : jb;          // baselines of one beam group, or all
    const long i = b * n_pol + p;
    const int nx = bln[2 * b], ny = bln[2 * b + 1];
    const int Bx = 2 * lg.H[0] + 1, K = lg.K;
    const cpx<G> *cellp = band + (((size_t)(lg.H[1] - ny) * Bx + (lg.H[0] - nx)) * K) * n_pol + p;
    cpx<double> v;
    if (wq == nullptr) {
        v = cmk<double>((double)cellp[0].x, (double)cellp[0].y);
    } else {
        v = cmk<double>(0.0, 0.0);
        for (int q = 0; q < K; ++q) {
            const cpx<G> t = cellp[(size_t)q * n_pol];
            v = cadd(v, cmul(wq[(size_t)b * K + q], cmk<double>((double)t.x, (double)t.y)));
        }
    }
    const double s = dx[nx + lg.H[0]] * dy[ny + lg.H[1]];
    if (out_fp64) {
        reinterpret_cast<cpx<double> *>(out)[i] = cmk<double>(v.x * s, v.y * s);
    } else {
        reinterpret_cast<cpx<float> *>(out)[i] = cmk<float>((float)(v.x * s), (float)(v.y * s));
    }
}

template <class G>
cudaError_t launch_gather_lattice(const cpx<G> *band, const int *bln, const int *bl_list, int n_bl, int n_pol,
                                  const LatGeom &lg, const cpx<double> *wq, const double *dx, const double *dy,
                                  void *out, int out_fp64, cudaStream_t st)
{
    const long n = (long)n_bl * n_pol;
    if (n <= 0) return cudaSuccess;
    k_gather_lattice<G><<<(unsigned)((n + 63) / 64), 64, 0, st>>>(band, bln, bl_list, n_bl, n_pol, lg, wq, dx, dy,
                                                                   out, out_fp64);
    return cudaGetLastError();
}

__global__ void k_lattice_wterms(const double *__restrict__ b_up, int n_bl, int K, double kappa,
                                 cpx<double> *__restrict__ wq)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)n_bl * K) return;
    const long b = i / K;
    const int q = (int)(i - b * K);
    const double beta = 0.5 * kappa * b_up[b];
    const double j = (q == 0 ? 1.0 : 2.0) * bessel_jq(q, beta);
    double sb, cb;
    sincos(beta, &sb, &cb);
    cpx<double> f = cmk<double>(cb * j, -sb * j);          // e^{-i beta} eps_q J_q
    for (int k = 0; k < (q & 3); ++k) f = cmk<double>(f.y, -f.x);   // times (-i)^q
    wq[i] = f;
}

cudaError_t launch_lattice_wterms(const double *b_up, int n_bl, int K, double kappa, cpx<double> *wq,
                                  cudaStream_t st)
{
    const long n = (long)n_bl * K;
    if (n <= 0) return cudaSuccess;
    k_lattice_wterms<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b_up, n_bl, K, kappa, wq);
    return cudaGetLastError();
}

// Phihat(k) = int_{-1}^{1} phi(z) cos(k z) dz by Gauss-Legendre quadrature on
// the sine-substituted nodes of the plan (FP64).
__global__ void k_lattice_deconv(double *tab, int H, int nf, int w, double beta, const double *gl_x,
                                 const double *gl_w, int nq)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > 2 * H) return;
    const double k = M_PI * w * (double)(j - H) / nf;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += gl_w[q] * lat_es_d(gl_x[q], beta) * cos(k * gl_x[q]);
    tab[j] = 1.0 / (0.5 * w * s);
}

cudaError_t launch_lattice_deconv(double *tab, int H, int nf, int w, double beta, const double *gl_x,
                                  const double *gl_w, int nq, cudaStream_t st)
{
    k_lattice_deconv<<<(2 * H + 1 + 127) / 128, 128, 0, st>>>(tab, H, nf, w, beta, gl_x, gl_w, nq);
    return cudaGetLastError();
}

template cudaError_t launch_prep_lattice<float>(const double *, const int *, const int *, long, const void *, int,
                                                int, int, const SliceGeom &, const LatGeom &, int *, float *,
                                                cpx<float> *, cudaStream_t);
template cudaError_t launch_prep_lattice<double>(const double *, const int *, const int *, long, const void *, int,
                                                 int, int, const SliceGeom &, const LatGeom &, int *, double *,
                                                 cpx<double> *, cudaStream_t);
template cudaError_t launch_spread_lattice<float>(const int *, const int *, const float *, const cpx<float> *, long,
                                                  const SliceGeom &, const LatGeom &, cpx<float> *, cudaStream_t);
template cudaError_t launch_spread_lattice<double>(const int *, const int *, const double *, const cpx<double> *,
                                                   long, const SliceGeom &, const LatGeom &, cpx<double> *,
                                                   cudaStream_t);
template cudaError_t launch_gather_lattice<float>(const cpx<float> *, const int *, const int *, int, int,
                                                  const LatGeom &, const cpx<double> *, const double *,
                                                  const double *, void *, int, cudaStream_t);
template cudaError_t launch_gather_lattice<double>(const cpx<double> *, const int *, const int *, int, int,
                                                   const LatGeom &, const cpx<double> *, const double *,
                                                   const double *, void *, int, cudaStream_t);

}  // namespace fv
