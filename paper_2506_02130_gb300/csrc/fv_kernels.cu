// Device kernels of the visibility path except the FFT passes:
// set-up tables, weighting + spreading, interpolation + deconvolution +
// postphase, output scatter.  See fv_internal.cuh for the notation.
#include "fv_internal.cuh"

#include <math.h>

namespace fv {

// Exponential-of-semicircle kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on
// [-1, 1], zero outside (Section 2.2, spreading step).
__device__ __forceinline__ double es_kernel(double z, double beta)
{
    double t = 1.0 - z * z;
    return t >= 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}
__device__ __forceinline__ float es_kernel(float z, float beta)
{
    float t = 1.0f - z * z;
    return t >= 0.0f ? expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}

// Two consecutive complex values in one vector load (the address is a multiple of 2 complex).
__device__ __forceinline__ void load_pair(const cpx<float> *p, cpx<float> &a, cpx<float> &b)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    a = cmk<float>(v.x, v.y);
    b = cmk<float>(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const cpx<double> *p, cpx<double> &a, cpx<double> &b)
{
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    a = cmk<double>(v0.x, v0.y);
    b = cmk<double>(v1.x, v1.y);
}

// Phihat(k) = int_{-1}^{1} phi(z) cos(k z) dz by Gauss-Legendre quadrature (FP64).
__device__ double es_fourier(double k, double beta, const double *gl_x, const double *gl_w, int nq)
{
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += gl_w[q] * es_kernel(gl_x[q], beta) * cos(k * gl_x[q]);
    return s;
}

// ------------------------------------------------------------------ set-up
__global__ void k_radec_to_unit(const double *ra, const double *dec, long n, double *e)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sa, ca, sd, cd;
    sincos(ra[i], &sa, &ca);
    sincos(dec[i], &sd, &cd);
    e[i] = cd * ca;
    e[n + i] = cd * sa;
    e[2 * n + i] = sd;
}

// out[f][n][k] = in[k][n][f] through a shared tile of 32 sources x 32 channels per Stokes parameter: reads
// run along channels, writes along (source, Stokes).
template <class T>
__global__ void __launch_bounds__(256) k_flux_transpose(const T *__restrict__ in, long n_src, int n_stokes, int n_freq,
                                                        T *__restrict__ out)
{
    __shared__ T tile[4][32][33];
    const long n0 = (long)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int k = 0; k < n_stokes; ++k)
        for (int r = ty; r < 32; r += 8) {
            const long n = n0 + r;
            const int f = f0 + tx;
            tile[k][r][tx] = (n < n_src && f < n_freq) ? in[((size_t)k * n_src + n) * n_freq + f] : (T)0;
        }
    __syncthreads();
    const int per = 32 * n_stokes;                  // (source, Stokes) values of one channel in the tile
    for (int c = 0; c < 32; ++c) {
        const int f = f0 + c;
        if (f >= n_freq) break;
        for (int v = threadIdx.x; v < per; v += blockDim.x) {
            const int r = v / n_stokes, k = v - r * n_stokes;
            const long n = n0 + r;
            if (n < n_src) out[((size_t)f * n_src + n) * n_stokes + k] = tile[k][r][c];
        }
    }
}

cudaError_t launch_flux_transpose(const void *flux, int fp64, long n_src, int n_stokes, int n_freq, void *out,
                                  cudaStream_t st)
{
    if (n_src <= 0 || n_freq <= 0) return cudaSuccess;
    if (n_stokes < 1 || n_stokes > 4) return cudaErrorInvalidValue;
    dim3 blocks((unsigned)((n_src + 31) / 32), (unsigned)((n_freq + 31) / 32));
    if (fp64)
        k_flux_transpose<double><<<blocks, 256, 0, st>>>((const double *)flux, n_src, n_stokes, n_freq, (double *)out);
    else
        k_flux_transpose<float><<<blocks, 256, 0, st>>>((const float *)flux, n_src, n_stokes, n_freq, (float *)out);
    return cudaGetLastError();
}

cudaError_t launch_radec_to_unit(const double *ra, const double *dec, long n, double *e, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_radec_to_unit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ra, dec, n, e);
    return cudaGetLastError();
}

__global__ void k_source_extents(const double *e, long n, const double *R_all, int n_time, double *out)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double ex = e[i], ey = e[n + i], ez = e[2 * n + i];
        for (int t = 0; t < n_time; ++t) {
            const double *R = R_all + 9 * t;
            double s2 = R[6] * ex + R[7] * ey + R[8] * ez;
            if (!(s2 > 0.0)) continue;
            double s0 = R[0] * ex + R[1] * ey + R[2] * ez;
            double s1 = R[3] * ex + R[4] * ey + R[5] * ez;
            lo[0] = fmin(lo[0], s0); hi[0] = fmax(hi[0], s0);
            lo[1] = fmin(lo[1], s1); hi[1] = fmax(hi[1], s1);
            lo[2] = fmin(lo[2], s2); hi[2] = fmax(hi[2], s2);
        }
    }
    __shared__ double red[6][256];
    for (int k = 0; k < 3; ++k) { red[k][threadIdx.x] = lo[k]; red[3 + k][threadIdx.x] = hi[k]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) {
                red[k][threadIdx.x] = fmin(red[k][threadIdx.x], red[k][threadIdx.x + s]);
                red[3 + k][threadIdx.x] = fmax(red[3 + k][threadIdx.x], red[3 + k][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_source_extents(const double *e, long n, const double *R_all, int n_time, double *out,
                                  int nblocks, cudaStream_t st)
{
    k_source_extents<<<nblocks, 256, 0, st>>>(e, n, R_all, n_time, out);
    return cudaGetLastError();
}

template <class G>
__global__ void k_prescale_table(G *tab, int nf1, int M, int w, double beta, const double *gl_x,
                                 const double *gl_w, int nq)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf1) return;
    double k = (double)(j - nf1 / 2) * w * M_PI / (double)M;
    tab[j] = (G)(1.0 / es_fourier(k, beta, gl_x, gl_w, nq));
}

template <class G>
cudaError_t launch_prescale_table(G *tab, int nf1, int M, int w, double beta, const double *gl_x,
                                  const double *gl_w, int nq, cudaStream_t st)
{
    k_prescale_table<G><<<(nf1 + 127) / 128, 128, 0, st>>>(tab, nf1, M, w, beta, gl_x, gl_w, nq);
    return cudaGetLastError();
}

template <class G>
__global__ void k_twiddles(cpx<G> *tw, int M)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)M, &s, &c);
    tw[k] = cmk<G>((G)c, (G)s);
}

template <class G>
cudaError_t launch_twiddles(cpx<G> *tw, int M, cudaStream_t st)
{
    k_twiddles<G><<<(M + 255) / 256, 256, 0, st>>>(tw, M);
    return cudaGetLastError();
}

__global__ void k_target_deconv(const double *bu, int n_u, int d, double bc0, double bc1, double bc2,
                                double bh0, double bh1, double bh2, int w, double beta, double sigma,
                                const double *gl_x, const double *gl_w, int nq, double *dec)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_u) return;
    const double bc[3] = {bc0, bc1, bc2}, bh[3] = {bh0, bh1, bh2};
    double r = 1.0;
    for (int i = 0; i < d; ++i) {
        double a = bh[i] > 0.0 ? (bc[i] - bu[3 * u + i]) / bh[i] * (w * M_PI / (2.0 * sigma)) : 0.0;
        r *= (4.0 / ((double)w * w)) / es_fourier(a, beta, gl_x, gl_w, nq);
    }
    dec[u] = r;
}

cudaError_t launch_target_deconv(const double *bu, int n_u, int d, const double *bcen, const double *bhalf,
                                 int w, double beta, double sigma, const double *gl_x, const double *gl_w,
                                 int nq, double *dec, cudaStream_t st)
{
    if (n_u <= 0) return cudaSuccess;
    k_target_deconv<<<(n_u + 127) / 128, 128, 0, st>>>(bu, n_u, d, bcen[0], bcen[1], bcen[2], bhalf[0],
                                                      bhalf[1], bhalf[2], w, beta, sigma, gl_x, gl_w, nq,
                                                      dec);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ weighting
__device__ __forceinline__ double load_flux(const void *flux, int fp64, size_t idx)
{
    return fp64 ? ((const double *)flux)[idx] : (double)((const float *)flux)[idx];
}

// Strengths c^{pq} = [J C J^dagger]_{pq} (Eq. 1-2) with J = A R(az):
// the rotation turns (Q, U) by twice the azimuth and leaves I and V alone.
__device__ __forceinline__ int source_strengths(const SliceGeom &g, const void *flux, int flux_fp64,
                                                long n_src, int n_freq, int f, long n, double s0, double s1,
                                                double s2, cpx<double> *c)
{
    double rho = sqrt(s0 * s0 + s1 * s1);
    double A = beam_voltage<double>(g.beam, s0, s1, rho, s2, g.nu, f);
    double A2 = g.two_beams ? A * beam_voltage<double>(g.beam2, s0, s1, rho, s2, g.nu, f) : A * A;
    const void *fl = g.flux_t ? g.flux_t : flux;
    double I = load_flux(fl, flux_fp64, flux_index(g, 0, n, n_src, n_freq, f));
    if (!g.polarized) {
        c[0] = cmk<double>(A2 * I, 0.0);
        return 1;
    }
    double Q = load_flux(fl, flux_fp64, flux_index(g, 1, n, n_src, n_freq, f));
    double U = load_flux(fl, flux_fp64, flux_index(g, 2, n, n_src, n_freq, f));
    double V = load_flux(fl, flux_fp64, flux_index(g, 3, n, n_src, n_freq, f));
    double ca = 1.0, sa = 0.0;
    if (rho > 0.0) { ca = s1 / rho; sa = s0 / rho; }
    double c2 = ca * ca - sa * sa, s2a = 2.0 * ca * sa;
    double Qr = Q * c2 - U * s2a, Ur = Q * s2a + U * c2;
    c[0] = cmk<double>(A2 * (I + Qr), 0.0);
    c[1] = cmk<double>(A2 * Ur, A2 * V);
    c[2] = cmk<double>(A2 * Ur, -A2 * V);
    c[3] = cmk<double>(A2 * (I - Qr), 0.0);
    return 4;
}

// ------------------------------------------------------------------ spreading
template <class G>
__global__ void __launch_bounds__(128) k_spread_direct(const double *__restrict__ e, long n_src,
                                                       const void *__restrict__ flux, int flux_fp64, int n_freq,
                                                       int f, SliceGeom g, cpx<G> *__restrict__ grid)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_src) return;
    const double ex = e[n], ey = e[n_src + n], ez = e[2 * n_src + n];
    const double s2 = g.R[6] * ex + g.R[7] * ey + g.R[8] * ez;
    if (!(s2 > 0.0)) return;                       // horizon cut (strictly above)
    const double s0 = g.R[0] * ex + g.R[1] * ey + g.R[2] * ez;
    const double s1 = g.R[3] * ex + g.R[4] * ey + g.R[5] * ez;
    cpx<double> c[4];
    const int np = source_strengths(g, flux, flux_fp64, n_src, n_freq, f, n, s0, s1, s2, c);
    // prephase e^{i D.(s - C)} (FP64)
    const double st[3] = {s0 - g.dim[0].C, s1 - g.dim[1].C, s2 - g.dim[2].C};
    double ph = 0.0;
    for (int i = 0; i < g.d; ++i) ph += g.dim[i].D * st[i];
    double sp, cp;
    sincos(ph, &sp, &cp);
    cpx<G> cg[4];
    for (int p = 0; p < np; ++p) {
        cpx<double> v = cmul(c[p], cmk<double>(cp, sp));
        cg[p] = cmk<G>((G)v.x, (G)v.y);
    }
    // kernel weights per dimension; the cell split of q is done in FP64
    G kv[3][16];
    int base[3] = {0, 0, 0};
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w;
    for (int i = 0; i < 3; ++i) {
        if (i >= g.d) { kv[i][0] = (G)1; base[i] = 0; continue; }
        double q = st[i] * g.dim[i].qscale;
        double l0 = ceil(q - 0.5 * w);
        G fr = (G)(l0 - q);                        // offset of cell l0 from q, in [-w/2, 1-w/2)
        for (int j = 0; j < w; ++j) kv[i][j] = es_kernel(two_over_w * (fr + (G)j), geom_beta<G>(g));
        int b = (int)l0 + g.dim[i].nf1 / 2;
        base[i] = b;
    }
    const int nx = g.dim[0].nf1, ny = g.dim[1].nf1, nz = g.d == 3 ? g.dim[2].nf1 : 1;
    const int wz = g.d == 3 ? w : 1;
    const size_t plane = (size_t)nx * ny * nz;
    for (int jz = 0; jz < wz; ++jz) {
        int iz = base[2] + jz;
        if (g.d == 3) { iz %= nz; if (iz < 0) iz += nz; }
        for (int jy = 0; jy < w; ++jy) {
            int iy = (base[1] + jy) % ny; if (iy < 0) iy += ny;
            G wyz = kv[2][g.d == 3 ? jz : 0] * kv[1][jy];
            for (int jx = 0; jx < w; ++jx) {
                int ix = (base[0] + jx) % nx; if (ix < 0) ix += nx;
                G wt = wyz * kv[0][jx];
                size_t idx = ((size_t)iz * ny + iy) * nx + ix;
                for (int p = 0; p < np; ++p) {
                    atomicAdd(&grid[p * plane + idx].x, cg[p].x * wt);
                    atomicAdd(&grid[p * plane + idx].y, cg[p].y * wt);
                }
            }
        }
    }
}

template <class G>
cudaError_t launch_spread_direct(const double *e, long n_src, const void *flux, int flux_fp64, int n_freq, int f,
                                 const SliceGeom &g, cpx<G> *grid, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    k_spread_direct<G><<<(unsigned)((n_src + 127) / 128), 128, 0, st>>>(e, n_src, flux, flux_fp64, n_freq, f, g,
                                                                         grid);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ interpolation
template <class G>
__global__ void __launch_bounds__(128) k_interp(const cpx<G> *__restrict__ band, const double *__restrict__ bu,
                                                int n_u, const double *__restrict__ dec, SliceGeom g,
                                                cpx<double> *__restrict__ Vu)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_u) return;
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w;
    double x[3] = {0.0, 0.0, 0.0};
    G kv[3][16];
    int base[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        if (i >= g.d) { kv[i][0] = (G)1; continue; }
        x[i] = -g.kappa * bu[3 * u + i];               // target x_k = -2 pi nu b_k / c
        double p = (x[i] - g.dim[i].D) * g.dim[i].pscale;
        double m0 = ceil(p - 0.5 * w);
        G fr = (G)(p - m0);                            // offset of p from cell m0, in (w/2-1, w/2]
        for (int j = 0; j < w; ++j) kv[i][j] = es_kernel(two_over_w * (fr - (G)j), geom_beta<G>(g));
        base[i] = (int)m0 + g.dim[i].H;
    }
    const int np = g.n_pol;
    const int Bx = g.dim[0].B, By = g.dim[1].B;
    const int wz = g.d == 3 ? w : 1;
    G acc[8];
    for (int k = 0; k < 2 * np; ++k) acc[k] = (G)0;
    for (int jz = 0; jz < wz; ++jz) {
        int bz = g.d == 3 ? base[2] + jz : 0;
        for (int jy = 0; jy < w; ++jy) {
            int by = base[1] + jy;
            G wyz = kv[2][g.d == 3 ? jz : 0] * kv[1][jy];
            const cpx<G> *row = band + (((size_t)bz * By + by) * Bx) * np;
            for (int jx = 0; jx < w; ++jx) {
                G wt = wyz * kv[0][jx];
                const cpx<G> *cell = row + (size_t)(base[0] + jx) * np;
                for (int p = 0; p < np; ++p) {
                    cpx<G> v = cell[p];
                    acc[2 * p] += wt * v.x;
                    acc[2 * p + 1] += wt * v.y;
                }
            }
        }
    }
    // deconvolution (FP64, channel independent) and postphase e^{i x.C} (FP64)
    double ph = 0.0;
    for (int i = 0; i < g.d; ++i) ph += x[i] * g.dim[i].C;
    double sp, cp;
    sincos(ph, &sp, &cp);
    const double dk = dec[u];
    for (int p = 0; p < np; ++p) {
        cpx<double> v = cmk<double>((double)acc[2 * p] * dk, (double)acc[2 * p + 1] * dk);
        Vu[(size_t)u * np + p] = cmul(v, cmk<double>(cp, sp));
    }
}

template <class G>
cudaError_t launch_interp(const cpx<G> *band, const double *bu, int n_u, const double *dec, const SliceGeom &g,
                          cpx<double> *Vu, cudaStream_t st)
{
    if (n_u <= 0) return cudaSuccess;
    k_interp<G><<<(n_u + 127) / 128, 128, 0, st>>>(band, bu, n_u, dec, g, Vu);
    return cudaGetLastError();
}

// Interpolation with the z axis evaluated directly (3-D transforms whose z
// grid is short, and 2-D transforms with Nz = 1).  The z FFT followed by the
// z interpolation of one target,
//     sum_{m_z in footprint} phi((2/w)(p_z - m_z)) sum_{l_z} a_{l_z} e^{2 pi i l_z m_z / M_z},
// is regrouped exactly as sum_{l_z} a_{l_z} K(l_z) with
//     K(l_z) = sum_{m_z} phi((2/w)(p_z - m_z)) e^{2 pi i l_z m_z / M_z},
// so the band after the x and y passes, [b_y][b_x][pol][l_z], is read with
// the z prescale folded into K.  One warp per target: the lanes split the
// w x w footprint in (y, x) and reduce with shuffles.  With height terms
// (g.K > 0) the band's l_z are the terms q and K(q) is the target's weight of
// term q (height_weight): the same sum.
template <class G, bool HASZ>
__global__ void __launch_bounds__(256) k_interp_zdirect(const cpx<G> *__restrict__ band, const double *__restrict__ bu,
                                                        int n_u, const double *__restrict__ dec, SliceGeom g,
                                                        const G *__restrict__ prez, const cpx<G> *__restrict__ twz,
                                                        cpx<double> *__restrict__ Vu)
{
    const int lane = threadIdx.x & 31;
    const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= n_u) return;
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w;
    const G beta = geom_beta<G>(g);
    double x[3] = {0.0, 0.0, 0.0};
    G fr[3];
    int m0[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        fr[i] = (G)0;
        if (i < g.d) {
            x[i] = -g.kappa * bu[3 * u + i];
            double p = (x[i] - g.dim[i].D) * g.dim[i].pscale;
            double m = ceil(p - 0.5 * w);
            m0[i] = (int)m;
            fr[i] = (G)(p - m);
        }
    }
    const int Nz = HASZ ? g.dim[2].nf1 : 1;
    // lane lz < Nz builds K(l_z); the vector is then shared through shuffles
    cpx<G> Kmine = cmk<G>((G)1, (G)0);
    if (HASZ && lane < Nz && g.K) {
        Kmine = height_weight<G>(g, bu[3 * u + 2], lane);     // height terms: the target's weights
    } else if (HASZ && lane < Nz) {
        const int Mz = g.dim[2].M;
        const int lc = lane - Nz / 2;
        cpx<G> acc = cmk<G>((G)0, (G)0);
        int e = (lc * m0[2]) % Mz;
        if (e < 0) e += Mz;
        int step = lc % Mz;
        if (step < 0) step += Mz;
        for (int jz = 0; jz < w; ++jz) {
            const G wt = es_kernel(two_over_w * (fr[2] - (G)jz), beta);
            acc = cadd(acc, cscale(twz[e], wt));
            e += step;
            if (e >= Mz) e -= Mz;
        }
        Kmine = cscale(acc, prez[lane]);
    }
    // the vector in registers: loops over it are unrolled to the largest Nz (16) with a guard, so that it is
    // never indexed dynamically
    cpx<G> K[HASZ ? 16 : 1];
    if (HASZ) {
#pragma unroll
        for (int lz = 0; lz < 16; ++lz) {
            K[lz].x = __shfl_sync(0xffffffffu, Kmine.x, lz);
            K[lz].y = __shfl_sync(0xffffffffu, Kmine.y, lz);
        }
    }
    const int np = g.n_pol;
    const int Bx = g.dim[0].B;
    const int bx0 = m0[0] + g.dim[0].H, by0 = m0[1] + g.dim[1].H;
    // x and y kernel values: lane j < w holds the j-th, the others read them by shuffle
    const G wxm = lane < w ? es_kernel(two_over_w * (fr[0] - (G)lane), beta) : (G)0;
    const G wym = lane < w ? es_kernel(two_over_w * (fr[1] - (G)lane), beta) : (G)0;
    G acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = (G)0;
    const bool vec2 = (Nz % 2) == 0;   // z runs of even length are read as pairs of complex values
    for (int base = 0; base < w * w; base += 32) {   // same trip count on every lane (shuffles)
        const int idx = base + lane;
        const bool valid = idx < w * w;
        const int jy = valid ? idx / w : 0, jx = valid ? idx - jy * w : 0;
        const G wt = __shfl_sync(0xffffffffu, wym, jy) * __shfl_sync(0xffffffffu, wxm, jx);
        if (valid) {
            const cpx<G> *cell = band + (((size_t)(by0 + jy) * Bx + (bx0 + jx)) * np) * Nz;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (p >= np) break;
                cpx<G> s = cmk<G>((G)0, (G)0);
                const cpx<G> *c = cell + p * Nz;
                if (!HASZ) {
                    s = c[0];
                } else if (vec2) {
#pragma unroll
                    for (int lz = 0; lz < (HASZ ? 16 : 1); lz += 2) {
                        if (lz < Nz) {
                            cpx<G> v0, v1;
                            load_pair(c + lz, v0, v1);
                            s = cadd(s, cadd(cmul(v0, K[lz]), cmul(v1, K[lz + 1])));
                        }
                    }
                } else {
#pragma unroll
                    for (int lz = 0; lz < (HASZ ? 16 : 1); ++lz)
                        if (lz < Nz) s = cadd(s, cmul(c[lz], K[lz]));
                }
                acc[2 * p] += wt * s.x;
                acc[2 * p + 1] += wt * s.y;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (k < 2 * np)   // np is uniform across the warp
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane == 0) {
        double ph = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < g.d) ph += x[i] * g.dim[i].C;
        double sp, cp;
        sincos(ph, &sp, &cp);
        const double dk = dec[u];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (p >= np) break;
            cpx<double> v = cmk<double>((double)acc[2 * p] * dk, (double)acc[2 * p + 1] * dk);
            Vu[(size_t)u * np + p] = cmul(v, cmk<double>(cp, sp));
        }
    }
}

// The same sum for one polarisation and a short, even z axis in FP32, read
// row by row: one warp per target, lane = c * (Nz/2) + h holds z values
// (2h, 2h+1) of footprint cell c of the current footprint row, so a warp
// reads one row of the footprint (w cells x Nz values, contiguous in the
// band) with a single 16-byte load per lane.  The lane applies K(2h),
// K(2h+1) and the row's y weight, scales by its cell's x weight at the end,
// and the warp reduces.  Needs w * Nz / 2 <= 32.
__global__ void __launch_bounds__(256) k_interp_zrow(const cpx<float> *__restrict__ band,
                                                     const double *__restrict__ bu, int n_u,
                                                     const double *__restrict__ dec, SliceGeom g,
                                                     const float *__restrict__ prez,
                                                     const cpx<float> *__restrict__ twz, cpx<double> *__restrict__ Vu)
{
    const int lane = threadIdx.x & 31;
    const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= n_u) return;
    const int w = g.w;
    const float two_over_w = 2.0f / (float)w;
    const float beta = g.beta_f;
    double x[3] = {0.0, 0.0, 0.0};
    float fr[3];
    int m0[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        fr[i] = 0.0f;
        if (i < g.d) {
            x[i] = -g.kappa * bu[3 * u + i];
            double p = (x[i] - g.dim[i].D) * g.dim[i].pscale;
            double m = ceil(p - 0.5 * w);
            m0[i] = (int)m;
            fr[i] = (float)(p - m);
        }
    }
    const int Nz = g.d == 3 || g.K ? g.dim[2].nf1 : 1;     // up planes or height terms
    const int L = Nz / 2;                    // lanes per footprint cell
    // K(l_z) for l_z = lane < Nz, as in k_interp_zdirect
    cpx<float> Kmine = cmk<float>(1.0f, 0.0f);
    if (lane < Nz && g.K) {
        Kmine = height_weight<float>(g, bu[3 * u + 2], lane);
    } else if (lane < Nz) {
        const int Mz = g.dim[2].M;
        const int lc = lane - Nz / 2;
        cpx<float> acc = cmk<float>(0.0f, 0.0f);
        int e = (lc * m0[2]) % Mz;
        if (e < 0) e += Mz;
        int step = lc % Mz;
        if (step < 0) step += Mz;
        for (int jz = 0; jz < w; ++jz) {
            const float wt = es_kernel(two_over_w * (fr[2] - (float)jz), beta);
            acc = cadd(acc, cscale(twz[e], wt));
            e += step;
            if (e >= Mz) e -= Mz;
        }
        Kmine = cscale(acc, prez[lane]);
    }
    const int c = lane / L, h = lane - c * L;
    const bool active = c < w;
    const int src = active ? 2 * h : 0;
    const cpx<float> K0 = cmk<float>(__shfl_sync(0xffffffffu, Kmine.x, src), __shfl_sync(0xffffffffu, Kmine.y, src));
    const cpx<float> K1 =
        cmk<float>(__shfl_sync(0xffffffffu, Kmine.x, src + 1), __shfl_sync(0xffffffffu, Kmine.y, src + 1));
    const float wxm = lane < w ? es_kernel(two_over_w * (fr[0] - (float)lane), beta) : 0.0f;
    const float wym = lane < w ? es_kernel(two_over_w * (fr[1] - (float)lane), beta) : 0.0f;
    const float wx = __shfl_sync(0xffffffffu, wxm, active ? c : 0);
    const int Bx = g.dim[0].B;
    const int bx0 = m0[0] + g.dim[0].H, by0 = m0[1] + g.dim[1].H;
    float ax = 0.0f, ay = 0.0f;
    for (int jy = 0; jy < w; ++jy) {        // same trip count on every lane (shuffle inside)
        const float wy = __shfl_sync(0xffffffffu, wym, jy);
        if (active) {
            const cpx<float> *cell = band + ((size_t)(by0 + jy) * Bx + (bx0 + c)) * Nz + 2 * h;
            cpx<float> v0, v1;
            load_pair(cell, v0, v1);
            const cpx<float> s = cadd(cmul(v0, K0), cmul(v1, K1));
            ax += wy * s.x;
            ay += wy * s.y;
        }
    }
    ax *= wx;
    ay *= wx;
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
        double ph = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < g.d) ph += x[i] * g.dim[i].C;
        double sp, cp;
        sincos(ph, &sp, &cp);
        const double dk = dec[u];
        const cpx<double> v = cmk<double>((double)ax * dk, (double)ay * dk);
        Vu[u] = cmul(v, cmk<double>(cp, sp));
    }
}

// Interpolation with the per-target set-up spread over the threads.  A CTA
// takes 32 targets: first threads 0-31 compute, one target each, the FP64
// coordinates, the first footprint cell, the kernel values of x and y (and
// for a short z axis the vector K(l_z) of the direct z sum), and the postphase
// and deconvolution factor, into shared memory.  Then each of the 4 warps
// walks 8 of the targets, all lanes reading footprint values from the band
// (ZROW: one footprint row of w cells x Nz z values per load round, one
// 16-byte load per lane; 2-D: lanes over the w x w cells, n_pol values each),
// and reduces; lane 0 writes the target's value.
constexpr int kIbThreads = 128;
constexpr int kIbTargets = 32;
constexpr int kIbPerWarp = kIbTargets / (kIbThreads / 32);
constexpr int kIbMaxW = 16;

template <class G, bool ZROW>
__global__ void __launch_bounds__(kIbThreads) k_interp_batch(const cpx<G> *__restrict__ band,
                                                             const double *__restrict__ bu, int n_u,
                                                             const double *__restrict__ dec, SliceGeom g,
                                                             const G *__restrict__ prez,
                                                             const cpx<G> *__restrict__ twz,
                                                             cpx<double> *__restrict__ Vu)
{
    __shared__ G s_wx[kIbTargets][kIbMaxW + 1], s_wy[kIbTargets][kIbMaxW + 1];
    __shared__ cpx<G> s_K[ZROW ? kIbTargets : 1][ZROW ? 8 : 1];
    __shared__ int s_bx[kIbTargets], s_by[kIbTargets];
    __shared__ cpx<double> s_post[kIbTargets];
    const long u0 = (long)blockIdx.x * kIbTargets;
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w, beta = geom_beta<G>(g);
    // --- per-target set-up, one target per thread
    if (threadIdx.x < kIbTargets) {
        const int tl = threadIdx.x;
        const long u = u0 + tl;
        const bool valid = u < n_u;
        double x[3] = {0.0, 0.0, 0.0};
        int m0[3] = {0, 0, 0};
        G fr[3] = {(G)0, (G)0, (G)0};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i < g.d && valid) {
                x[i] = -g.kappa * bu[3 * u + i];
                const double pp = (x[i] - g.dim[i].D) * g.dim[i].pscale;
                const double m = ceil(pp - 0.5 * w);
                m0[i] = (int)m;
                fr[i] = (G)(pp - m);
            }
        }
        for (int j = 0; j < w; ++j) {
            s_wx[tl][j] = es_kernel(two_over_w * (fr[0] - (G)j), beta);
            s_wy[tl][j] = es_kernel(two_over_w * (fr[1] - (G)j), beta);
        }
        s_bx[tl] = m0[0] + g.dim[0].H;
        s_by[tl] = m0[1] + g.dim[1].H;
        if (ZROW && g.K) {
            // height terms: the weights are computed by all threads below
        } else if (ZROW) {
            const int Nz = g.dim[2].nf1, Mz = g.dim[2].M;
            G phz[kIbMaxW];
#pragma unroll
            for (int jz = 0; jz < kIbMaxW; ++jz)
                phz[jz] = jz < w ? es_kernel(two_over_w * (fr[2] - (G)jz), beta) : (G)0;
            for (int lz = 0; lz < Nz; ++lz) {
                const int lc = lz - Nz / 2;
                int e = (lc * m0[2]) % Mz;
                if (e < 0) e += Mz;
                int step = lc % Mz;
                if (step < 0) step += Mz;
                cpx<G> acc = cmk<G>((G)0, (G)0);
#pragma unroll
                for (int jz = 0; jz < kIbMaxW; ++jz) {
                    if (jz < w) {
                        acc = cadd(acc, cscale(twz[e], phz[jz]));
                        e += step;
                        if (e >= Mz) e -= Mz;
                    }
                }
                s_K[ZROW ? tl : 0][ZROW ? lz : 0] = cscale(acc, prez[lz]);
            }
        }
        cpx<double> post = cmk<double>(0.0, 0.0);
        if (valid) {
            double ph = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (i < g.d) ph += x[i] * g.dim[i].C;
            double sp, cp;
            sincos(ph, &sp, &cp);
            post = cmk<double>(cp * dec[u], sp * dec[u]);
        }
        s_post[tl] = post;
    }
    if (ZROW && g.K) {
        // height weights of the CTA's targets, one (target, term) pair per thread and round
        const int Nz = g.dim[2].nf1;
        for (int idx = threadIdx.x; idx < kIbTargets * Nz; idx += kIbThreads) {
            const int tl = idx / Nz, lz = idx - tl * Nz;
            const long u = u0 + tl;
            s_K[ZROW ? tl : 0][ZROW ? lz : 0] = u < n_u ? height_weight<G>(g, bu[3 * u + 2], lz) : cmk<G>((G)0, (G)0);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = g.n_pol;
    const int Bx = g.dim[0].B;
    const int t0 = warp * kIbPerWarp;
    const int nt = (int)max(0L, min((long)kIbPerWarp, (long)n_u - u0 - t0));
    if (ZROW) {
        const int Nz = g.dim[2].nf1, L = Nz / 2;
        const int c = lane / L, h = lane - c * L;
        const bool active = c < w;
        const size_t rstride = (size_t)Bx * Nz;
        for (int tt = 0; tt < nt; ++tt) {
            const int t = t0 + tt;
            G ax = (G)0, ay = (G)0;
            if (active) {
                const cpx<G> K0 = s_K[ZROW ? t : 0][ZROW ? 2 * h : 0];
                const cpx<G> K1 = s_K[ZROW ? t : 0][ZROW ? 2 * h + 1 : 0];
                const cpx<G> *rowp = band + ((size_t)s_by[t] * Bx + (s_bx[t] + c)) * Nz + 2 * h;
#pragma unroll 4
                for (int jy = 0; jy < w; ++jy) {
                    cpx<G> v0, v1;
                    load_pair(rowp + jy * rstride, v0, v1);
                    const cpx<G> sm = cadd(cmul(v0, K0), cmul(v1, K1));
                    const G wy = s_wy[t][jy];
                    ax += wy * sm.x;
                    ay += wy * sm.y;
                }
                const G wx = s_wx[t][c];
                ax *= wx;
                ay *= wx;
            }
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (lane == 0) Vu[u0 + t] = cmul(cmk<double>((double)ax, (double)ay), s_post[t]);
        }
    } else {
        const int ww = w * w;
        for (int tt = 0; tt < nt; ++tt) {
            const int t = t0 + tt;
            G acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = (G)0;
            const int bx0 = s_bx[t], by0 = s_by[t];
            for (int idx = lane; idx < ww; idx += 32) {
                const int jy = idx / w, jx = idx - jy * w;
                const G wt = s_wx[t][jx] * s_wy[t][jy];
                const cpx<G> *cell = band + ((size_t)(by0 + jy) * Bx + (bx0 + jx)) * np;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    if (p < np) {
                        const cpx<G> v = cell[p];
                        acc[2 * p] += wt * v.x;
                        acc[2 * p + 1] += wt * v.y;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < 2 * np)   // np is the same on every lane
                    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (lane == 0) {
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    if (p < np)
                        Vu[(size_t)(u0 + t) * np + p] =
                            cmul(cmk<double>((double)acc[2 * p], (double)acc[2 * p + 1]), s_post[t]);
            }
        }
    }
}

// 2-D interpolation with one warp per target.  Lane 0 computes the target's FP64 quantities (coordinate
// on the FFT grid, first footprint cell, offset, postphase argument reduced to [-pi, pi]); lanes
// (dx, j) = (lane / J, lane % J), J = 32 / w, then cover footprint column dx and, with four products,
// product group j (each lane walks every row), or with one product, row group j.  A footprint row of a
// product group is one coalesced load (w cells x n_pol values contiguous in the band).  The sums over
// columns (and row groups) are shuffle reductions; the postphase sine and cosine run in the grid
// precision after the FP64 reduction of their argument.
template <class G, int NP>
__global__ void __launch_bounds__(256) k_interp_warp(const cpx<G> *__restrict__ band, const double *__restrict__ bu,
                                                     int n_u, const double *__restrict__ dec, SliceGeom g,
                                                     cpx<double> *__restrict__ Vu, SliceOut so)
{
    const int lane = threadIdx.x & 31;
    const long u = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= n_u) return;   // whole warps
    const int w = g.w;
    const G two_over_w = (G)2 / (G)w, beta = geom_beta<G>(g);
    int m0 = 0, m1 = 0;
    G f0 = (G)0, f1 = (G)0, phr = (G)0;
    if (sizeof(G) == 4 && g.tgt_db) {
        // FP32 set-up on every lane, no FP64: double-float products of the per-channel factors and the
        // target's float pairs, then the first footprint cell m = ceil(p - w/2) and f = p - m brought into
        // (w/2 - 1, w/2] (as the FP64 form), and the postphase reduced by 2 pi = 6.2831855 - 1.7484555e-7
        const float4 db = g.tgt_db[u];
        const float2 bc = g.tgt_bc[u];
        const float hw = 0.5f * (float)w;
        float mm[2], ff[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float dh = i == 0 ? db.x : db.z, dl = i == 0 ? db.y : db.w;
            float ph = g.a_hi[i] * dh;
            float pl = fmaf(g.a_hi[i], dh, -ph) + (g.a_hi[i] * dl + g.a_lo[i] * dh);
            ph = -ph;
            pl = -pl;                                   // p = ph + pl
            float m = ceilf(ph - hw);
            float f = (ph - m) + pl;
            if (f > hw) { m += 1.0f; f -= 1.0f; }
            else if (f <= hw - 1.0f) { m -= 1.0f; f += 1.0f; }
            mm[i] = m;
            ff[i] = f;
        }
        m0 = (int)mm[0];
        m1 = (int)mm[1];
        f0 = (G)ff[0];
        f1 = (G)ff[1];
        float qh = g.kap_hi * bc.x;
        const float ql = fmaf(g.kap_hi, bc.x, -qh) + (g.kap_hi * bc.y + g.kap_lo * bc.x);
        qh = -qh;                                        // argument -kappa (b . C) = qh - ql
        const float k = rintf(qh * 0.15915494f);
        phr = (G)(fmaf(-k, -1.7484555e-7f, fmaf(-k, 6.2831855f, qh)) - ql);
    } else if (lane == 0) {
        // FP64 set-up on lane 0
        double ph = 0.0;
        double fr[2];
        int mm[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double x = -g.kappa * bu[3 * u + i];
            const double pp = (x - g.dim[i].D) * g.dim[i].pscale;
            const double m = ceil(pp - 0.5 * w);
            mm[i] = (int)m;
            fr[i] = pp - m;
            ph += x * g.dim[i].C;
        }
        m0 = mm[0];
        m1 = mm[1];
        f0 = (G)fr[0];
        f1 = (G)fr[1];
        ph -= 6.283185307179586476925 * rint(ph * 0.15915494309189533577);
        phr = (G)ph;
    }
    if (!(sizeof(G) == 4 && g.tgt_db)) {
        m0 = __shfl_sync(0xffffffffu, m0, 0);
        m1 = __shfl_sync(0xffffffffu, m1, 0);
        f0 = __shfl_sync(0xffffffffu, f0, 0);
        f1 = __shfl_sync(0xffffffffu, f1, 0);
    }
    const int J = 32 / w;
    const int dx = lane / J, j = lane - dx * J;
    const bool on = dx < w;
    // this lane's x weight, and the y weight of row r held by lane r * J (shuffled per row)
    const G wx = on ? es_kernel(two_over_w * (f0 - (G)dx), beta) : (G)0;
    const G wyl = on ? es_kernel(two_over_w * (f1 - (G)dx), beta) : (G)0;
    const int Bx = g.dim[0].B;
    const cpx<G> *col = band + ((size_t)(m1 + g.dim[1].H) * Bx + (m0 + g.dim[0].H + (on ? dx : 0))) * NP;
    G ax[NP > 1 ? 4 : 1], ay[NP > 1 ? 4 : 1];
#pragma unroll
    for (int p = 0; p < (NP > 1 ? 4 : 1); ++p) ax[p] = ay[p] = (G)0;
    for (int r = 0; r < w; ++r) {
        const G wy = __shfl_sync(0xffffffffu, wyl, r * J);
        if (NP == 1) {
            if (on && r % J == j) {
                const cpx<G> v = col[(size_t)r * Bx];
                ax[0] += wy * v.x;
                ay[0] += wy * v.y;
            }
        } else if (on) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int pp = j + q * J;
                if (q * J < NP && pp < NP) {
                    const cpx<G> v = col[(size_t)r * Bx * NP + pp];
                    ax[q] += wy * v.x;
                    ay[q] += wy * v.y;
                }
            }
        }
    }
    const G phs = (sizeof(G) == 4 && g.tgt_db) ? phr : __shfl_sync(0xffffffffu, phr, 0);
    G sp, cp;
    if (sizeof(G) == 4) {
        float a, b;
        sincosf((float)phs, &a, &b);
        sp = (G)a;
        cp = (G)b;
    } else {
        // the FP64 path keeps the argument's FP64 reduction and an FP64 sine and cosine
        double a, b;
        sincos((double)phs, &a, &b);
        sp = (G)a;
        cp = (G)b;
    }
    const double dd = dec[u];
    if (so.out) {
        // the scatter fused in: every lane gets the target's NP values (in the grid precision) and the warp
        // writes them to the target's baselines, out[b][p]
        const G ddg = (G)dd;
        G rx[NP], ry[NP];
        if (NP == 1) {
            G x = ax[0] * wx, y = ay[0] * wx;
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                y += __shfl_xor_sync(0xffffffffu, y, o);
            }
            rx[0] = (x * cp - y * sp) * ddg;
            ry[0] = (x * sp + y * cp) * ddg;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q * J >= NP) break;   // uniform
                G x = ax[q] * wx, y = ay[q] * wx;
                for (int o = J; o < 32; o <<= 1) {
                    const G tx = __shfl_down_sync(0xffffffffu, x, o), ty = __shfl_down_sync(0xffffffffu, y, o);
                    if (lane + o < 32) {
                        x += tx;
                        y += ty;
                    }
                }
                const G fx = (x * cp - y * sp) * ddg, fy = (x * sp + y * cp) * ddg;
                // product pp of this group sits on lane pp - q J (column 0)
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                    const int src = pp - q * J;
                    const bool mine = src >= 0 && src < J;
                    const G vx = __shfl_sync(0xffffffffu, fx, mine ? src : 0);
                    const G vy = __shfl_sync(0xffffffffu, fy, mine ? src : 0);
                    if (mine) {
                        rx[pp] = vx;
                        ry[pp] = vy;
                    }
                }
            }
        }
        const int gu = so.u_base + (int)u;
        const int b0 = so.u_off[gu], nb = so.u_off[gu + 1] - b0;
        cpx<G> *o = reinterpret_cast<cpx<G> *>(so.out);
        for (int k = lane; k < nb * NP; k += 32) {
            const int kb = NP == 1 ? k : k >> 2, p = NP == 1 ? 0 : k & 3;
            G vx = rx[0], vy = ry[0];
#pragma unroll
            for (int q = 1; q < NP; ++q)
                if (p == q) {
                    vx = rx[q];
                    vy = ry[q];
                }
            o[(size_t)so.u_bl[b0 + kb] * NP + p] = cmk<G>(vx, vy);
        }
        return;
    }
    if (NP == 1) {
        G x = ax[0] * wx, y = ay[0] * wx;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) Vu[u] = cmk<double>(((double)x * cp - (double)y * sp) * dd, ((double)x * sp + (double)y * cp) * dd);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (q * J >= NP) break;   // uniform
            G x = ax[q] * wx, y = ay[q] * wx;
            // sum over the columns: lanes with the same j are J apart; a partner past lane 31 adds nothing
            // (a shuffle from there returns the caller's own value)
            for (int o = J; o < 32; o <<= 1) {
                const G tx = __shfl_down_sync(0xffffffffu, x, o), ty = __shfl_down_sync(0xffffffffu, y, o);
                if (lane + o < 32) {
                    x += tx;
                    y += ty;
                }
            }
            const int pp = j + q * J;
            if (dx == 0 && pp < NP)
                Vu[(size_t)u * NP + pp] =
                    cmk<double>(((double)x * cp - (double)y * sp) * dd, ((double)x * sp + (double)y * cp) * dd);
        }
    }
}

static bool zrow_fits(const SliceGeom &g, int elem_bytes)
{
    if (elem_bytes != 4 || (g.d != 3 && g.K == 0) || g.n_pol != 1) return false;
    const int Nz = g.dim[2].nf1;
    return Nz >= 2 && Nz % 2 == 0 && g.w * (Nz / 2) <= 32;
}

bool interp_fuses_scatter(const SliceGeom &g)
{
    return g.w <= kIbMaxW && g.d == 2 && g.K == 0 && (g.n_pol == 1 || g.n_pol == 4);
}

template <class G>
cudaError_t launch_interp_zdirect(const cpx<G> *band, const double *bu, int n_u, const double *dec,
                                  const SliceGeom &g, const G *prez, const cpx<G> *twz, cpx<double> *Vu,
                                  cudaStream_t st, const SliceOut *so)
{
    if (so && so->out && !interp_fuses_scatter(g)) return cudaErrorInvalidValue;
    const SliceOut sov = so ? *so : SliceOut{nullptr, nullptr, nullptr, 0};
    if (n_u <= 0) return cudaSuccess;
    if ((g.d == 3 || g.K) && g.dim[2].nf1 > 16) return cudaErrorInvalidValue;
    long threads = (long)n_u * 32;
    const unsigned ib_blocks = (unsigned)((n_u + kIbTargets - 1) / kIbTargets);
    if (g.w <= kIbMaxW) {
        if (g.d == 2 && g.K == 0) {
            // one warp per target, 8 per CTA
            const unsigned wb = (unsigned)((n_u + 7) / 8);
            if (g.n_pol == 4)
                k_interp_warp<G, 4><<<wb, 256, 0, st>>>(band, bu, n_u, dec, g, Vu, sov);
            else
                k_interp_warp<G, 1><<<wb, 256, 0, st>>>(band, bu, n_u, dec, g, Vu, sov);
            return cudaGetLastError();
        }
        if constexpr (sizeof(G) == 4) {
            if (zrow_fits(g, 4) && g.dim[2].nf1 <= 8) {
                k_interp_batch<G, true><<<ib_blocks, kIbThreads, 0, st>>>(band, bu, n_u, dec, g, prez, twz, Vu);
                return cudaGetLastError();
            }
            if (zrow_fits(g, 4)) {
                k_interp_zrow<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(band, bu, n_u, dec, g, prez, twz,
                                                                                Vu);
                return cudaGetLastError();
            }
        }
    }
    if (g.d == 3 || g.K)
        k_interp_zdirect<G, true><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(band, bu, n_u, dec, g, prez, twz,
                                                                                     Vu);
    else
        k_interp_zdirect<G, false><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(band, bu, n_u, dec, g, prez,
                                                                                      twz, Vu);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ output
__global__ void k_scatter(const cpx<double> *__restrict__ Vu, const int *__restrict__ bl2u, int n_bl, int n_pol,
                          void *out, int out_fp64)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)n_bl * n_pol) return;
    int bl = (int)(i / n_pol), p = (int)(i % n_pol);
    cpx<double> v = Vu[(size_t)bl2u[bl] * n_pol + p];
    if (out_fp64) ((double2 *)out)[i] = make_double2(v.x, v.y);
    else ((float2 *)out)[i] = make_float2((float)v.x, (float)v.y);
}

cudaError_t launch_scatter(const cpx<double> *Vu, const int *bl2u, int n_bl, int n_pol, void *out, int out_fp64,
                           cudaStream_t st)
{
    long n = (long)n_bl * n_pol;
    if (n <= 0) return cudaSuccess;
    k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Vu, bl2u, n_bl, n_pol, out, out_fp64);
    return cudaGetLastError();
}

// explicit instantiations
template cudaError_t launch_prescale_table<double>(double *, int, int, int, double, const double *, const double *,
                                                   int, cudaStream_t);
template cudaError_t launch_prescale_table<float>(float *, int, int, int, double, const double *, const double *,
                                                  int, cudaStream_t);
template cudaError_t launch_twiddles<double>(cpx<double> *, int, cudaStream_t);
template cudaError_t launch_twiddles<float>(cpx<float> *, int, cudaStream_t);
template cudaError_t launch_spread_direct<double>(const double *, long, const void *, int, int, int,
                                                  const SliceGeom &, cpx<double> *, cudaStream_t);
template cudaError_t launch_spread_direct<float>(const double *, long, const void *, int, int, int,
                                                 const SliceGeom &, cpx<float> *, cudaStream_t);
template cudaError_t launch_interp<double>(const cpx<double> *, const double *, int, const double *,
                                           const SliceGeom &, cpx<double> *, cudaStream_t);
template cudaError_t launch_interp_zdirect<double>(const cpx<double> *, const double *, int, const double *,
                                                   const SliceGeom &, const double *, const cpx<double> *,
                                                   cpx<double> *, cudaStream_t, const SliceOut *);
template cudaError_t launch_interp_zdirect<float>(const cpx<float> *, const double *, int, const double *,
                                                  const SliceGeom &, const float *, const cpx<float> *,
                                                  cpx<double> *, cudaStream_t, const SliceOut *);
template cudaError_t launch_interp<float>(const cpx<float> *, const double *, int, const double *,
                                          const SliceGeom &, cpx<double> *, cudaStream_t);

}  // namespace fv
