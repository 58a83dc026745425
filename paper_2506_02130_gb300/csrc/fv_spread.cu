// Binned, tiled ES-kernel spreading (Section 2.2, step 1).
//
// Per time (shared by every channel of that time):
//   k_bin_count    rotate equatorial -> ENU (Section 2.3), cut the horizon, and
//                  count the visible sources per tile of the top channel's grid;
//   k_bin_scan     exclusive scan of the counts (one CTA);
//   k_bin_scatter  counting-sort the visible directions by tile.
// Per (time, channel) slice:
//   k_prep         beam x flux strengths (Eq. 1-3), prephase e^{i D.(s-C)}
//                  with the argument and its 2 pi reduction in FP64, and the
//                  grid coordinate q = (s - C) sigma X / pi split in FP64 into
//                  the first footprint cell (int) and an offset (FP32 or FP64);
//   k_spread_gather one CTA per output tile: every thread owns (x, y) columns
//                  of the tile and adds, in registers, the sources whose
//                  footprint covers them (their records copied into shared
//                  memory by bulk asynchronous copies, chunk by chunk, double
//                  buffered, with their kernel values computed there), then
//                  stores its cells once.  Every grid cell is written by
//                  exactly one thread, so the grid needs no clearing and
//                  there are no atomics.
// A channel's grid coordinates are the top channel's scaled by r = qscale_f /
// qscale_top <= 1 per axis, so a tile of channel f maps to a rectangle of top
// bins, i.e. one contiguous range of sorted sources per bin row.
#include "fv_staged.cuh"
#include "fv_internal.cuh"

#include <math.h>

namespace fv {

// ------------------------------------------------------------------ per time
__global__ void k_bin_count(const double *__restrict__ e, long n_src, TimeBin tb, int *__restrict__ bin_of,
                            int *__restrict__ counts)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_src) return;
    const double ex = e[n], ey = e[n_src + n], ez = e[2 * n_src + n];
    const double s2 = tb.R[6] * ex + tb.R[7] * ey + tb.R[8] * ez;
    if (!(s2 > 0.0)) {
        bin_of[n] = -1;
        return;
    }
    const double s0 = tb.R[0] * ex + tb.R[1] * ey + tb.R[2] * ez;
    const double s1 = tb.R[3] * ex + tb.R[4] * ey + tb.R[5] * ez;
    int cx = top_cell((s0 - tb.C[0]) * tb.qscale_top[0], tb.nf1_top[0]);
    int cy = top_cell((s1 - tb.C[1]) * tb.qscale_top[1], tb.nf1_top[1]);
    int b = (cy / tb.T[1]) * tb.nbx + cx / tb.T[0];
    bin_of[n] = b;
    // warp-aggregated count: one atomic per distinct bin among the active lanes
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, b);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&counts[b], __popc(grp));
}

// exclusive scan of counts[0..nb) into offsets[0..nb], cursor = offsets (one CTA of 1024 threads)
__global__ void k_bin_scan(const int *__restrict__ counts, int nb, int *__restrict__ offsets, int *__restrict__ cursor)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int lo = t * per, hi = min(nb, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;   // exclusive prefix of this thread's chunk
    for (int i = lo; i < hi; ++i) {
        offsets[i] = run;
        cursor[i] = run;
        run += counts[i];
    }
    if (t == 1023) offsets[nb] = part[1023];
}

// Two floats hi + lo holding an FP64 value to about 2^-48 of its magnitude.
__device__ __forceinline__ float2 split_f2(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__global__ void k_bin_scatter(const double *__restrict__ e, long n_src, TimeBin tb, const int *__restrict__ bin_of,
                              int *__restrict__ cursor, double *__restrict__ sdir, int *__restrict__ sidx,
                              float4 *__restrict__ tc)
{
    long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (n >= n_src) return;
    const int b = bin_of[n];
    if (b < 0) return;
    // warp-aggregated slot reservation: the lowest lane of each group of equal bins reserves for all
    const int lane = threadIdx.x & 31;
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, b);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[b], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    const int pos = base + __popc(grp & ((1u << lane) - 1u));
    const double ex = e[n], ey = e[n_src + n], ez = e[2 * n_src + n];
    const double s[3] = {tb.R[0] * ex + tb.R[1] * ey + tb.R[2] * ez, tb.R[3] * ex + tb.R[4] * ey + tb.R[5] * ez,
                         tb.R[6] * ex + tb.R[7] * ey + tb.R[8] * ez};
    sdir[pos] = s[0];
    sdir[n_src + pos] = s[1];
    sdir[2 * n_src + pos] = s[2];
    sidx[pos] = (int)n;
    if (tc) {
        // the top channel's grid coordinates and prephase, in FP64, kept as float pairs: every channel's
        // are these times kappa / kappa_top
        double q[3] = {0.0, 0.0, 0.0}, ph = 0.0;
        for (int k = 0; k < tb.d; ++k) {
            const double st = s[k] - tb.C[k];
            q[k] = st * tb.qscale_top[k];
            ph += tb.D_top[k] * st;
        }
        const float2 qx = split_f2(q[0]), qy = split_f2(q[1]), qz = split_f2(q[2]), pp = split_f2(ph);
        tc[3 * (size_t)pos] = make_float4(qx.x, qx.y, qy.x, qy.y);
        tc[3 * (size_t)pos + 1] = make_float4(qz.x, qz.y, pp.x, pp.y);
        tc[3 * (size_t)pos + 2] = make_float4((float)s[0], (float)s[1], (float)s[2], 0.0f);
    }
}

cudaError_t launch_time_binning(const double *e, long n_src, const TimeBin &tb, int *bin_of, int *counts,
                                int *offsets, int *cursor, double *sdir, int *sidx, float4 *tc, cudaStream_t st)
{
    const int nb = tb.nbx * tb.nby;
    cudaError_t err = cudaMemsetAsync(counts, 0, (size_t)nb * sizeof(int), st);
    if (err != cudaSuccess) return err;
    if (n_src > 0) k_bin_count<<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(e, n_src, tb, bin_of, counts);
    k_bin_scan<<<1, 1024, 0, st>>>(counts, nb, offsets, cursor);
    if (n_src > 0)
        k_bin_scatter<<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(e, n_src, tb, bin_of, cursor, sdir, sidx,
                                                                       tc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per slice
// Strengths with prephase and the split grid coordinates of the sorted visible sources.  STAGED: written
// as staged records (rec[i], cs[i * stride + p]); otherwise as cell[3][n_src], frac[3][n_src],
// cs[n_pol][n_src].
template <class G, bool STAGED>
__global__ void __launch_bounds__(256) k_prep(const double *__restrict__ sdir, const int *__restrict__ sidx,
                                              const int *__restrict__ nv_ptr, long n_src,
                                              const void *__restrict__ flux, int flux_fp64, int n_freq, int f,
                                              SliceGeom g, int *__restrict__ cell, G *__restrict__ frac,
                                              cpx<G> *__restrict__ cs, SrcRec<G> *__restrict__ rec)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= *nv_ptr) return;
    const double s0 = sdir[i], s1 = sdir[n_src + i], s2 = sdir[2 * n_src + i];
    const long n = sidx[i];
    cpx<G> c[4];
    const int np = source_strengths<G>(g, s0, s1, s2, n, flux, flux_fp64, n_src, n_freq, f, c);
    // prephase: argument and reduction to [-pi, pi] in FP64, sincos in G
    const double st[3] = {s0 - g.dim[0].C, s1 - g.dim[1].C, s2 - g.dim[2].C};
    double ph = 0.0;
    for (int k = 0; k < g.d; ++k) ph += g.dim[k].D * st[k];
    ph -= 6.283185307179586476925 * rint(ph * 0.15915494309189533577);
    G sp, cp;
    if (sizeof(G) == 4) { float a, b; sincosf((float)ph, &a, &b); sp = (G)a; cp = (G)b; }
    else { double a, b; sincos(ph, &a, &b); sp = (G)a; cp = (G)b; }
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (p < np)
            cs[STAGED ? (size_t)i * staged_cs_stride((int)sizeof(G), np) + p : (size_t)p * n_src + i] =
                cmul(c[p], cmk<G>(cp, sp));
    // grid coordinates: first footprint cell l0 = ceil(q - w/2) and offset l0 - q of q = (s - C) qscale,
    // the product in FP64.  FP64 grids split in FP64; FP32 grids split q into q_hi + q_lo (floats, q_lo
    // the FP64 remainder) and take l0 and l0 - q_hi in FP32, exact but where q_hi - w/2 rounds onto an
    // integer, which moves the footprint by one cell and drops a kernel value below e^-beta
    int ci[3] = {0, 0, 0};
    G fr[3] = {(G)0, (G)0, (G)0};
    for (int k = 0; k < 3; ++k) {
        if (k < g.d) {
            const double q = st[k] * g.dim[k].qscale;
            if (sizeof(G) == 4) {
                const float qh = (float)q, ql = (float)(q - (double)qh);
                const float l0 = ceilf(qh - 0.5f * (float)g.w);
                ci[k] = (int)l0 + g.dim[k].nf1 / 2;
                fr[k] = (G)((l0 - qh) - ql);
            } else {
                const double l0 = ceil(q - 0.5 * g.w);
                ci[k] = (int)l0 + g.dim[k].nf1 / 2;
                fr[k] = (G)(l0 - q);
            }
            // Eq. 5 keeps every footprint inside the grid; a rounding at its very edge moves the footprint
            // back in by one cell (the offset follows, l0 - q stays exact)
            const int hi = g.dim[k].nf1 - g.w;
            if (ci[k] < 0) {
                fr[k] -= (G)ci[k];
                ci[k] = 0;
            } else if (ci[k] > hi) {
                fr[k] -= (G)(ci[k] - hi);
                ci[k] = hi;
            }
        }
    }
    if (g.K) fr[2] = (G)((s2 - g.hc) / g.hs);     // height terms: the argument u of T_q (no up grid axis)
    if (STAGED) {
        SrcRec<G> h;
        h.cell = (unsigned)ci[0] | ((unsigned)ci[1] << 14) | ((unsigned)ci[2] << 28);
        h.fx = fr[0];
        h.fy = fr[1];
        h.fz = fr[2];
        rec[i] = h;
    } else {
        for (int k = 0; k < 3; ++k) {
            cell[(size_t)k * n_src + i] = ci[k];
            frac[(size_t)k * n_src + i] = fr[k];
        }
    }
}

// FP32 grids: the same strengths, prephase and grid coordinates from the per-time records tc (see
// launch_time_binning) without FP64 arithmetic.  Every channel's coordinate and prephase are the top
// channel's times r = kappa / kappa_top, formed in double-float arithmetic (an exact product by FMA plus
// the cross terms, about 2^-44 relative); the prephase is reduced by 2 pi split in two floats; the first
// footprint cell follows from the accurate offset l0 - q, which is brought into [-w/2, 1 - w/2).
__device__ __forceinline__ float2 mul_df(float ah, float al, float bh, float bl)
{
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p) + (ah * bl + al * bh);
    return make_float2(p, e);
}

// One source of one slice from its per-time record (a, b, sd) and source index n: strengths with prephase
// c[0..np), first footprint cells ci and offsets fr.
struct PrepOne {
    cpx<float> c[4];
    int np;
    int ci[3];
    float fr[3];
};

__device__ __forceinline__ void prep_tc_one(const float4 a, const float4 b, const float4 sd, long n, const void *flux,
                                            int flux_fp64, long n_src, int n_freq, int f, const SliceGeom &g,
                                            PrepOne &o)
{
    o.np = source_strengths<float, float>(g, sd.x, sd.y, sd.z, n, flux, flux_fp64, n_src, n_freq, f, o.c);
    // prephase r ph_top, reduced to about [-pi, pi]: 2 pi = 6.2831855 - 1.7484555e-7
    const float2 ph = mul_df(g.rsc_hi, g.rsc_lo, b.z, b.w);
    const float k = rintf(ph.x * 0.15915494f);
    const float phr = fmaf(-k, -1.7484555e-7f, fmaf(-k, 6.2831855f, ph.x)) + ph.y;
    float sp, cp;
    sincosf(phr, &sp, &cp);
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (p < o.np) o.c[p] = cmul(o.c[p], cmk<float>(cp, sp));
    const float hw = 0.5f * (float)g.w;
#pragma unroll
    for (int k3 = 0; k3 < 3; ++k3) {
        o.ci[k3] = 0;
        o.fr[k3] = 0.0f;
        if (k3 < g.d) {
            const float qh = k3 == 0 ? a.x : (k3 == 1 ? a.z : b.x), ql = k3 == 0 ? a.y : (k3 == 1 ? a.w : b.y);
            const float2 q = mul_df(g.rsc_hi, g.rsc_lo, qh, ql);
            float l0 = ceilf(q.x - hw);
            float off = (l0 - q.x) - q.y;                 // l0 - q
            if (off >= 1.0f - hw) { l0 -= 1.0f; off -= 1.0f; }
            else if (off < -hw) { l0 += 1.0f; off += 1.0f; }
            int c = (int)l0 + g.dim[k3].nf1 / 2;
            const int hi = g.dim[k3].nf1 - g.w;
            if (c < 0) { off -= (float)c; c = 0; }
            else if (c > hi) { off -= (float)(c - hi); c = hi; }
            o.ci[k3] = c;
            o.fr[k3] = off;
        }
    }
    if (g.K) o.fr[2] = (sd.z - g.hc_f) * g.hs_inv_f;    // height terms: the argument u of T_q
}

// MODE 0: cell / frac / cs arrays; 1: staged records
template <int MODE>
__global__ void __launch_bounds__(256) k_prep_tc(const float4 *__restrict__ tc, const int *__restrict__ sidx,
                                                 const int *__restrict__ nv_ptr, long n_src,
                                                 const void *__restrict__ flux, int flux_fp64, int n_freq, int f,
                                                 SliceGeom g, int *__restrict__ cell, float *__restrict__ frac,
                                                 cpx<float> *__restrict__ cs, SrcRec<float> *__restrict__ rec)
{
    constexpr bool STAGED = MODE > 0;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= *nv_ptr) return;
    PrepOne o;
    prep_tc_one(tc[3 * i], tc[3 * i + 1], tc[3 * i + 2], sidx[i], flux, flux_fp64, n_src, n_freq, f, g, o);
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (p < o.np) cs[STAGED ? (size_t)i * staged_cs_stride(4, o.np) + p : (size_t)p * n_src + i] = o.c[p];
    if (STAGED) {
        SrcRec<float> h;
        h.cell = (unsigned)o.ci[0] | ((unsigned)o.ci[1] << 14) | ((unsigned)o.ci[2] << 28);
        h.fx = o.fr[0];
        h.fy = o.fr[1];
        h.fz = o.fr[2];
        rec[i] = h;
    } else {
        for (int k3 = 0; k3 < 3; ++k3) {
            cell[(size_t)k3 * n_src + i] = o.ci[k3];
            frac[(size_t)k3 * n_src + i] = o.fr[k3];
        }
    }
}

// Ring records (the ring gather of two-dimensional grids): the same per source plus the footprint's
// kernel values.  A CTA's 256 sources are contiguous in the sorted order, so their per-time records are
// read into shared memory and their ring records and strengths written out of it with coalesced 16-byte
// accesses (each thread's own 48-byte read and 80 + 32-byte writes would touch a sector per lane).
template <int NP>
__global__ void __launch_bounds__(256) k_prep_ring(const float4 *__restrict__ tc, const int *__restrict__ sidx,
                                                   const int *__restrict__ nv_ptr, long n_src,
                                                   const void *__restrict__ flux, int flux_fp64, int n_freq, int f,
                                                   SliceGeom g, cpx<float> *__restrict__ cs,
                                                   RingRec *__restrict__ ring_rec, int *__restrict__ tile_ctr)
{
    constexpr int kCsw = (NP * 8 + 15) / 16 * 16 / 8;            // strengths per source, 16-byte rows
    constexpr int kRec4 = (int)(sizeof(RingRec) / sizeof(float4)), kCs4 = kCsw / 2;
    __shared__ float4 s_in[256 * 3];
    __shared__ float4 s_rec[256 * kRec4];
    __shared__ float4 s_cs[256 * kCs4];
    if (tile_ctr && blockIdx.x == 0 && threadIdx.x < 4) tile_ctr[threadIdx.x] = 0;
    const long i0 = (long)blockIdx.x * 256;
    const long nv = *nv_ptr;
    if (i0 >= nv) return;                                       // the same on every thread of the CTA
    const int cnt = (int)min(256L, nv - i0);
    for (int k = threadIdx.x; k < cnt * 3; k += 256) s_in[k] = tc[3 * i0 + k];
    __syncthreads();
    const int t = threadIdx.x;
    if (t < cnt) {
        PrepOne o;
        prep_tc_one(s_in[3 * t], s_in[3 * t + 1], s_in[3 * t + 2], sidx[i0 + t], flux, flux_fp64, n_src, n_freq, f,
                    g, o);
        RingRec h;
        h.cell = (unsigned)o.ci[0] | ((unsigned)o.ci[1] << 14);
        h.pad = 0u;
        const float two_over_w = 2.0f / (float)g.w, beta = g.beta_f;
#pragma unroll
        for (int j = 0; j <= kRingWmax; ++j) {
            h.wx[j] = j < g.w ? es_kernel_f(two_over_w * (o.fr[0] + (float)j), beta) : 0.0f;
            h.wy[j] = j < g.w ? es_kernel_f(two_over_w * (o.fr[1] + (float)j), beta) : 0.0f;
        }
        reinterpret_cast<RingRec *>(s_rec)[t] = h;
        cpx<float> *sc = reinterpret_cast<cpx<float> *>(s_cs) + (size_t)t * kCsw;
#pragma unroll
        for (int p = 0; p < kCsw; ++p) sc[p] = p < NP ? o.c[p] : cmk<float>(0.0f, 0.0f);
    }
    __syncthreads();
    float4 *gr = reinterpret_cast<float4 *>(ring_rec + i0);
    for (int k = threadIdx.x; k < cnt * kRec4; k += 256) gr[k] = s_rec[k];
    float4 *gc = reinterpret_cast<float4 *>(cs + (size_t)i0 * kCsw);
    for (int k = threadIdx.x; k < cnt * kCs4; k += 256) gc[k] = s_cs[k];
}

cudaError_t launch_prep_tc(const float4 *tc, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                           int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, float *frac,
                           cpx<float> *cs, SrcRec<float> *rec, RingRec *ring_rec, int *tile_ctr, cudaStream_t st)
{
    if (n_src <= 0) return tile_ctr ? cudaErrorInvalidValue : cudaSuccess;
    if (ring_rec && (g.w > kRingWmax || g.d != 2 || g.K || (g.n_pol != 1 && g.n_pol != 4)))
        return cudaErrorInvalidValue;
    const unsigned nb = (unsigned)((n_src + 255) / 256);
    if (ring_rec) {
        if (g.n_pol == 4)
            k_prep_ring<4><<<nb, 256, 0, st>>>(tc, sidx, nv_ptr, n_src, flux, flux_fp64, n_freq, f, g, cs, ring_rec,
                                               tile_ctr);
        else
            k_prep_ring<1><<<nb, 256, 0, st>>>(tc, sidx, nv_ptr, n_src, flux, flux_fp64, n_freq, f, g, cs, ring_rec,
                                               tile_ctr);
    } else if (rec) {
        k_prep_tc<1><<<nb, 256, 0, st>>>(tc, sidx, nv_ptr, n_src, flux, flux_fp64, n_freq, f, g, cell, frac, cs,
                                         rec);
    } else {
        k_prep_tc<0><<<nb, 256, 0, st>>>(tc, sidx, nv_ptr, n_src, flux, flux_fp64, n_freq, f, g, cell, frac, cs,
                                         rec);
    }
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_prep(const double *sdir, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                        int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, G *frac, cpx<G> *cs,
                        cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    k_prep<G, false><<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(sdir, sidx, nv_ptr, n_src, flux, flux_fp64,
                                                                      n_freq, f, g, cell, frac, cs, nullptr);
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_prep_staged(const double *sdir, const int *sidx, const int *nv_ptr, long n_src,
                               const void *flux, int flux_fp64, int n_freq, int f, const SliceGeom &g,
                               SrcRec<G> *rec, cpx<G> *cs, cudaStream_t st)
{
    if (n_src <= 0) return cudaSuccess;
    k_prep<G, true><<<(unsigned)((n_src + 255) / 256), 256, 0, st>>>(sdir, sidx, nv_ptr, n_src, flux, flux_fp64,
                                                                     n_freq, f, g, nullptr, nullptr, cs, rec);
    return cudaGetLastError();
}

// Gather form of the tiled spreading.  A CTA of 8 warps owns a 32 x 8 tile
// of (x, y) columns; warp k owns an 8 x 4 patch of it and each lane one
// column, holding that column's NZ z cells and NP products in registers.  The
// tile's candidate sources (bins of 8 x 4 top-channel cells) are staged in
// shared memory in chunks: per source its x and y kernel values, its z kernel
// values placed at absolute z (zero elsewhere) and its strengths.  While
// staging, each source is appended to the candidate list of every patch its
// footprint overlaps (shared-memory integer atomics); each warp then adds the
// sources of its own list.  No float atomics; every grid cell is stored once.
constexpr int kGatherThreads = 256;
constexpr int kWmax = 16;
constexpr int kWpad = kWmax + 1;            // row stride of the staged x/y kernel values (bank spread)
constexpr int kPatchX = 8, kPatchY = 4;     // one warp
constexpr int kTileX = 32, kTileY = 8;      // one CTA (4 x 2 patches)
constexpr int kPatches = 8;

// resident CTAs per SM the register allocation must allow without spills (fewer when the complex
// accumulators of a lane take 48 registers or more: 24 complex sums in FP32, 12 in FP64)
template <class G, int NP, int NZ> struct GatherMinBlocks {
    static constexpr int value = NP * NZ * (int)sizeof(G) >= 96 ? 2 : 4;
};

// REC: the candidates come as staged records (rec[i], strengths cs[i * stride + p], written by
// launch_prep_staged); thread 0 copies each chunk's ranges into shared memory with bulk asynchronous
// copies, double buffered, so that the next chunk arrives while the current one is added.  Otherwise
// every thread loads its candidate from cell[3][n], frac[3][n], cs[n_pol][n].
template <class G, int NP, int NZ, bool REC>
__global__ void __launch_bounds__(kGatherThreads, (GatherMinBlocks<G, NP, NZ>::value)) k_spread_gather(const int *__restrict__ offsets,
                                                                  const int *__restrict__ cell,
                                                                  const G *__restrict__ frac,
                                                                  const cpx<G> *__restrict__ cs, long n_src,
                                                                  SliceGeom g, TimeBin tb, double r0, double r1,
                                                                  const SrcRec<G> *__restrict__ rec,
                                                                  int *__restrict__ status,
                                                                  cpx<G> *__restrict__ grid)
{
    // candidates staged per round: 128 (96 in FP64, to keep the static shared memory under 48 KB)
    constexpr int kGatherChunk = sizeof(G) == 8 ? 96 : 128;
    constexpr int kCsw = REC ? (NP * 2 * (int)sizeof(G) + 15) / 16 * 16 / (2 * (int)sizeof(G)) : NP;
    __shared__ int s_cz[NZ > 1 ? kGatherChunk : 1];
    __shared__ G s_fx[kGatherChunk], s_fy[kGatherChunk], s_fz[NZ > 1 ? kGatherChunk : 1];
    // x kernel values (3-D), or for 2-D grids the strengths already weighted by them: s_cwx[(t w + dx) NP + p]
    // = c_p(t) psi_x(t, dx) in dynamic shared memory (kGatherChunk x w x NP complex values)
    // and the y kernel values s_wy[t * w + j], after them (2-D) or alone (3-D)
    constexpr bool CWX = NZ == 1;
    __shared__ G s_wx[CWX ? 1 : kGatherChunk * kWpad];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    cpx<G> *s_cwx = reinterpret_cast<cpx<G> *>(s_dyn);
    G *s_wy = reinterpret_cast<G *>(s_dyn + (CWX ? (size_t)kGatherChunk * g.w * NP * sizeof(cpx<G>) : 0));
    __shared__ __align__(16) G s_wz[NZ > 1 ? kGatherChunk : 1][NZ];
    __shared__ cpx<G> s_c[REC ? 1 : NP][REC ? 1 : kGatherChunk];
    // record staging (REC): two buffers of [records][strengths], their barriers and sizes
    __shared__ __align__(16) SrcRec<G> s_rec[REC ? 2 : 1][REC ? kGatherChunk : 1];
    __shared__ __align__(16) cpx<G> s_cs[REC ? 2 : 1][REC ? kGatherChunk * kCsw : 1];
    __shared__ __align__(8) uint64_t s_bar[2];
    // patch lists: candidate t (bits 0-7) with its footprint origin relative to the tile, cx - x0 + 16
    // (bits 8-15) and cy - y0 + 16 (bits 16-23), so that one shared load gives all three
    __shared__ __align__(16) int s_list[kPatches][kGatherChunk];
    __shared__ int s_cnt[kPatches];
    __shared__ int s_row0[32], s_pre[32], s_total;
    const int nx = g.dim[0].nf1, ny = g.dim[1].nf1, nz = g.d == 3 || g.K ? g.dim[2].nf1 : 1;
    const int w = g.w;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = x0 + (warp & 3) * kPatchX, py0 = y0 + (warp >> 2) * kPatchY;   // this warp's patch
    const int gx = px0 + (lane & 7), gy = py0 + (lane >> 3);                         // this lane's column
    cpx<G> acc[NP][NZ];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int z = 0; z < NZ; ++z) acc[p][z] = cmk<G>((G)0, (G)0);
    if (threadIdx.x < kPatches) s_cnt[threadIdx.x] = 0;
    // sources whose footprint can meet this tile (one-cell margin through the top-grid mapping): the bin
    // rectangle, computed once per CTA in FP64 by one thread (GB300's FP64 rate is a sixty-fourth of FP32)
    __shared__ int s_bins[4];
    if (threadIdx.x == 0) {
        const double qx_lo = (x0 - nx / 2 - 0.5 * w) / r0, qx_hi = (x0 + kTileX - nx / 2 + 0.5 * w - 1) / r0;
        const double qy_lo = (y0 - ny / 2 - 0.5 * w) / r1, qy_hi = (y0 + kTileY - ny / 2 + 0.5 * w - 1) / r1;
        s_bins[0] = top_cell(qx_lo - 1.0, tb.nf1_top[0]) / tb.T[0];
        s_bins[1] = top_cell(qx_hi + 1.0, tb.nf1_top[0]) / tb.T[0];
        s_bins[2] = top_cell(qy_lo - 1.0, tb.nf1_top[1]) / tb.T[1];
        s_bins[3] = top_cell(qy_hi + 1.0, tb.nf1_top[1]) / tb.T[1];
        if (REC) {
            mbar_init1(&s_bar[0]);
            mbar_init1(&s_bar[1]);
        }
    }
    const G two_over_w = (G)2 / (G)w, beta = geom_beta<G>(g);
    // floor(v / w) for v < kGatherChunk * kWmax by a float product: (v + 0.5) / w lies at least 1/(2w) from
    // an integer, far more than the product's rounding error
    const float inv_w = 1.0f / (float)w;
    __syncthreads();
    const int bx_lo = s_bins[0], bx_hi = s_bins[1], by_lo = s_bins[2], by_hi = s_bins[3];
    bool ok = true;
    unsigned phase = 0u;   // REC: bit b = parity of the next completion of buffer b's barrier
    int kc = 0;            // REC: chunks consumed (buffer kc & 1)
    // REC, thread 0: copy candidates [base, base + n) of the current rows table into buffer b
    auto issue = [&](int b, int base, int n, int nrows) {
        mbar_expect(&s_bar[b], (unsigned)n * (unsigned)(sizeof(SrcRec<G>) + kCsw * sizeof(cpx<G>)));
        for (int r = 0; r < nrows; ++r) {
            const int len = (r + 1 < nrows ? s_pre[r + 1] : s_total) - s_pre[r];
            const int a = max(base, s_pre[r]), e = min(base + n, s_pre[r] + len);
            if (a >= e) continue;
            const int i0 = s_row0[r] + (a - s_pre[r]), m = e - a;
            bulk_g2s(&s_rec[b][a - base], rec + i0, (unsigned)(m * sizeof(SrcRec<G>)), &s_bar[b]);
            bulk_g2s(&s_cs[b][(a - base) * kCsw], cs + (size_t)i0 * kCsw, (unsigned)(m * kCsw * sizeof(cpx<G>)),
                     &s_bar[b]);
        }
    };
    // The candidates of the tile are the bins [bx_lo, bx_hi] of the rows [by_lo, by_hi]: one contiguous
    // range of the sorted sources per row.  Rows are taken 32 at a time; their ranges are concatenated
    // (lengths scanned by warp 0) and cut into full chunks, so that a chunk is not limited to one row.
    for (int r0w = by_lo; r0w <= by_hi && ok; r0w += 32) {
        const int nrows = min(32, by_hi - r0w + 1);
        if (warp == 0) {
            int start = 0, len = 0;
            if (lane < nrows) {
                const int row = (r0w + lane) * tb.nbx;
                start = offsets[row + bx_lo];
                len = offsets[row + bx_hi + 1] - start;
            }
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            s_row0[lane] = start;
            s_pre[lane] = incl - len;
            if (lane == 31) s_total = incl;
            __syncwarp();
            if (REC && lane == 0 && s_total > 0) issue(kc & 1, 0, min(kGatherChunk, s_total), nrows);
        }
        __syncthreads();
        const int total = s_total;
        for (int base = 0; base < total; base += kGatherChunk, ++kc) {
            const int n = min(kGatherChunk, total - base);
            const int b = kc & 1;
            if (REC) {
                // the next chunk goes into the other buffer, which every thread finished with
                if (threadIdx.x == 0 && base + kGatherChunk < total)
                    issue(b ^ 1, base + kGatherChunk, min(kGatherChunk, total - base - kGatherChunk), nrows);
                const bool got = mbar_wait(&s_bar[b], (phase >> b) & 1u);
                phase ^= 1u << b;
                if (__syncthreads_or(!got)) {
                    // a copy did not arrive in time: record it, let thread 0 wait (bounded) for the copy it
                    // issued into the other buffer, and store zeros
                    ok = false;
                    if (threadIdx.x == 0) {
                        atomicOr(status, FV_DEVICE_TIMEOUT);
                        if (base + kGatherChunk < total) mbar_wait(&s_bar[b ^ 1], (phase >> (b ^ 1)) & 1u);
                    }
                    break;
                }
            }
            // 1. one thread per candidate: position, strengths, and the patches its footprint overlaps
            if (threadIdx.x < n) {
                const int t = threadIdx.x;
                int cx, cy;
                if (REC) {
                    const SrcRec<G> rr = s_rec[b][t];
                    cx = (int)(rr.cell & 0x3fffu);
                    cy = (int)((rr.cell >> 14) & 0x3fffu);
                    s_fx[t] = rr.fx;
                    s_fy[t] = rr.fy;
                    if (g.d == 3 || g.K) {
                        s_cz[NZ > 1 ? t : 0] = (int)(rr.cell >> 28);
                        s_fz[NZ > 1 ? t : 0] = rr.fz;
                    }
                } else {
                    const int v = base + threadIdx.x;
                    // the row holding the v-th candidate: the last row whose prefix is <= v
                    int r = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (r + step < nrows && s_pre[r + step] <= v) r += step;
                    const int i = s_row0[r] + (v - s_pre[r]);
                    cx = cell[i];
                    cy = cell[n_src + i];
                    s_fx[t] = frac[i];
                    s_fy[t] = frac[n_src + i];
                    if (g.d == 3 || g.K) {
                        s_cz[NZ > 1 ? t : 0] = cell[2 * n_src + i];
                        s_fz[NZ > 1 ? t : 0] = frac[2 * n_src + i];
                    }
#pragma unroll
                    for (int p = 0; p < NP; ++p) s_c[REC ? 0 : p][REC ? 0 : t] = cs[(size_t)p * n_src + i];
                }
                const int ax = max(cx - x0, 0), bx = min(cx + w - 1 - x0, kTileX - 1);
                const int ay = max(cy - y0, 0), by2 = min(cy + w - 1 - y0, kTileY - 1);
                if (ax <= bx && ay <= by2) {
                    for (int qy = ay / kPatchY; qy <= by2 / kPatchY; ++qy)
                        for (int qx = ax / kPatchX; qx <= bx / kPatchX; ++qx) {
                            const int q = qy * 4 + qx;
                            const int pos = atomicAdd(&s_cnt[q], 1);
                            s_list[q][pos] = t | ((cx - x0 + 16) << 8) | ((cy - y0 + 16) << 16);
                        }
                }
            }
            __syncthreads();
            // 2. every thread computes kernel values: x and y values (source, j), then z values placed at
            //    absolute z (zero outside the footprint)
            for (int v = threadIdx.x; v < n * w; v += kGatherThreads) {
                const int t = (int)(((float)v + 0.5f) * inv_w);
                const int j = v - t * w;
                const G ex = es_k<G>(two_over_w * (s_fx[t] + (G)j), beta);
                if (CWX) {
                    cpx<G> cw[NP];
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        cw[p] = cscale(REC ? s_cs[b][t * kCsw + p] : s_c[REC ? 0 : p][REC ? 0 : t], ex);
                    if (NP == 4 && sizeof(G) == 4) {
                        // entry v holds two 16-byte halves, stored swapped when bit 2 of v is set: the eight
                        // consecutive entries one list entry's lanes read then fall on distinct banks
                        const int sw = (v >> 2) & 1;
                        float4 *dst = reinterpret_cast<float4 *>(s_cwx + (size_t)v * NP);
                        dst[sw] = make_float4((float)cw[0].x, (float)cw[0].y, (float)cw[NP > 1 ? 1 : 0].x,
                                              (float)cw[NP > 1 ? 1 : 0].y);
                        dst[sw ^ 1] = make_float4((float)cw[NP > 2 ? 2 : 0].x, (float)cw[NP > 2 ? 2 : 0].y,
                                                  (float)cw[NP > 3 ? 3 : 0].x, (float)cw[NP > 3 ? 3 : 0].y);
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) s_cwx[(size_t)v * NP + p] = cw[p];
                    }
                } else {
                    s_wx[CWX ? 0 : t * kWpad + j] = ex;
                }
                s_wy[v] = es_k<G>(two_over_w * (s_fy[t] + (G)j), beta);   // v = t * w + j
            }
            if (NZ > 1 && g.K) {
                // height terms: plane q takes T_q(u) (three-term recurrence), zero for q >= K
                for (int t = threadIdx.x; t < n; t += kGatherThreads) {
                    const G u = s_fz[t];
                    G tm = (G)1, tq = u;
                    s_wz[t][0] = (G)1;
#pragma unroll
                    for (int q = 1; q < NZ; ++q) {
                        s_wz[t][q] = q < g.K ? tq : (G)0;
                        const G tn = (G)2 * u * tq - tm;
                        tm = tq;
                        tq = tn;
                    }
                }
            } else if (NZ > 1) {
                for (int v = threadIdx.x; v < n * NZ; v += kGatherThreads) {
                    const int t = v / NZ, z = v % NZ;
                    const int jz = z - s_cz[t];
                    s_wz[t][z] = (jz >= 0 && jz < w) ? es_k<G>(two_over_w * (s_fz[t] + (G)jz), beta) : (G)0;
                }
            }
            __syncthreads();
            // 3. each warp adds the sources of its patch list into its lanes' columns
            const int cnt = s_cnt[warp];
            const int lx16 = gx - x0 + 16, ly16 = gy - y0 + 16;
            if (CWX) {
                // 2-D: acc_p += psi_y(dy) (c_p psi_x(dx)), the weighted strengths of footprint column dx.
                // Four list entries per round, without branches (a lane outside a footprint adds a zero
                // weight times a valid table entry), so that their shared-memory loads overlap.
                cpx<G> acc2[NP];   // a second set of sums for alternate entries (independent FMA chains)
#pragma unroll
                for (int p = 0; p < NP; ++p) acc2[p] = cmk<G>((G)0, (G)0);
                auto one = [&](int ent, cpx<G> *sum) {
                    const int t = ent & 0xff;
                    const unsigned dx = (unsigned)(lx16 - ((ent >> 8) & 0xff)), dy = (unsigned)(ly16 - (ent >> 16));
                    const bool in = dx < (unsigned)w && dy < (unsigned)w;
                    const int cx = in ? (int)dx : 0, cy = in ? (int)dy : 0;
                    const G wy = in ? s_wy[t * w + cy] : (G)0;
                    const int ve = t * w + cx;
                    const cpx<G> *cw = s_cwx + (size_t)ve * NP;
                    cpx<G> v[NP];
                    if (NP == 4 && sizeof(G) == 4) {
                        const int sw = (ve >> 2) & 1;   // the halves' swizzle (see the table's stores)
                        const float4 a = reinterpret_cast<const float4 *>(cw)[sw];
                        const float4 c = reinterpret_cast<const float4 *>(cw)[sw ^ 1];
                        v[0] = cmk<G>((G)a.x, (G)a.y);
                        v[NP > 1 ? 1 : 0] = cmk<G>((G)a.z, (G)a.w);
                        v[NP > 2 ? 2 : 0] = cmk<G>((G)c.x, (G)c.y);
                        v[NP > 3 ? 3 : 0] = cmk<G>((G)c.z, (G)c.w);
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) v[p] = cw[p];
                    }
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        sum[p].x += wy * v[p].x;
                        sum[p].y += wy * v[p].y;
                    }
                };
                cpx<G> acc1[NP];
#pragma unroll
                for (int p = 0; p < NP; ++p) acc1[p] = acc[p][0];
                int e = 0;
                for (; e + 8 <= cnt; e += 8) {
                    const int4 qa = *reinterpret_cast<const int4 *>(&s_list[warp][e]);
                    const int4 qb = *reinterpret_cast<const int4 *>(&s_list[warp][e + 4]);
                    one(qa.x, acc1);
                    one(qa.y, acc2);
                    one(qa.z, acc1);
                    one(qa.w, acc2);
                    one(qb.x, acc1);
                    one(qb.y, acc2);
                    one(qb.z, acc1);
                    one(qb.w, acc2);
                }
                for (; e < cnt; ++e) one(s_list[warp][e], (e & 1) ? acc2 : acc1);
#pragma unroll
                for (int p = 0; p < NP; ++p) acc[p][0] = cadd(acc1[p], acc2[p]);
            }
            for (int e = 0; !CWX && e < cnt; ++e) {
                const int ent = s_list[warp][e];
                const int t = ent & 0xff;
                const unsigned dx = (unsigned)(lx16 - ((ent >> 8) & 0xff)), dy = (unsigned)(ly16 - (ent >> 16));
                if (dx < (unsigned)w && dy < (unsigned)w) {
                    const G wxy = s_wx[CWX ? 0 : t * kWpad + dx] * s_wy[t * w + dy];
                    G wz[NZ];
                    if (NZ > 1) {
#pragma unroll
                        for (int z = 0; z < NZ; ++z) wz[z] = s_wz[t][z];
                    } else {
                        wz[0] = (G)1;
                    }
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const cpx<G> cp = cscale(REC ? s_cs[b][t * kCsw + p] : s_c[REC ? 0 : p][REC ? 0 : t], wxy);
#pragma unroll
                        for (int z = 0; z < NZ; ++z) {
                            acc[p][z].x += cp.x * wz[z];
                            acc[p][z].y += cp.y * wz[z];
                        }
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x < kPatches) s_cnt[threadIdx.x] = 0;
            __syncthreads();
        }
        __syncthreads();      // every thread has read s_total before warp 0 rewrites the row table
    }
    if (gx < nx && gy < ny) {
        // the x and y prescale of the FFT passes, applied here once per cell when the plan asks for it
        const G sc = ok ? (g.pre_x ? ((const G *)g.pre_x)[gx] * ((const G *)g.pre_y)[gy] : (G)1) : (G)0;
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int z = 0; z < NZ; ++z)
                if (z < nz) grid[(((size_t)p * nz + z) * ny + gy) * nx + gx] = cscale(acc[p][z], sc);
    }
}

template <class G, int NP, int NZ>
static cudaError_t gather_launch(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                 const SliceGeom &g, const TimeBin &tb, double r0, double r1,
                                 const SrcRec<G> *rec, int *status, cpx<G> *grid, cudaStream_t st)
{
    constexpr int kChunkG = sizeof(G) == 8 ? 96 : 128;
    // dynamic shared memory: the weighted strengths (2-D) and the y kernel values, kChunkG x w each
    const size_t per_w = (NZ == 1 ? NP * sizeof(cpx<G>) : 0) + sizeof(G);
    const size_t dyn = (size_t)kChunkG * g.w * per_w;
    static bool attr_set[64][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int ri = rec ? 1 : 0;
    if (!attr_set[dev][ri]) {
        const void *fn = rec ? (const void *)k_spread_gather<G, NP, NZ, true> : (const void *)k_spread_gather<G, NP, NZ, false>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kChunkG * kWmax * per_w));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set[dev][ri] = true;
    }
    dim3 blocks((g.dim[0].nf1 + kTileX - 1) / kTileX, (g.dim[1].nf1 + kTileY - 1) / kTileY);
    if (rec)
        k_spread_gather<G, NP, NZ, true><<<blocks, kGatherThreads, dyn, st>>>(offsets, cell, frac, cs, n_src, g, tb,
                                                                              r0, r1, rec, status, grid);
    else
        k_spread_gather<G, NP, NZ, false><<<blocks, kGatherThreads, dyn, st>>>(offsets, cell, frac, cs, n_src, g, tb,
                                                                               r0, r1, rec, status, grid);
    return cudaGetLastError();
}

int spread_gather_config(int elem_bytes, int n_pol, int nz, int w, int *nz_tmpl, int *bin_x, int *bin_y)
{
    if (w > kWmax) return 0;
    const int NZ = nz <= 1 ? 1 : (nz <= 8 ? 8 : (nz <= 12 ? 12 : (nz <= 16 ? 16 : 0)));
    if (NZ == 0) return 0;
    const int budget = elem_bytes == 4 ? 32 : 16;       // complex accumulators per lane
    if (n_pol * NZ > budget) return 0;
    *nz_tmpl = NZ;
    *bin_x = kPatchX;
    *bin_y = kPatchY;
    return 1;
}

// The gather kernel for a slice: candidates from cell/frac/cs (rec == nullptr) or from staged records.
template <class G>
static cudaError_t gather_dispatch(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                   const SliceGeom &g, const TimeBin &tb, double r0, double r1, const SrcRec<G> *rec,
                                   int *status, cpx<G> *grid, cudaStream_t st)
{
    const int nz = g.d == 3 || g.K ? g.dim[2].nf1 : 1;     // up planes or height terms
    int NZ = 0, bx = 0, by = 0;
    if (!spread_gather_config(sizeof(G), g.n_pol, nz, g.w, &NZ, &bx, &by)) return cudaErrorInvalidValue;
    const int key = (g.n_pol == 4 ? 100 : 0) + NZ;
#define FV_GATHER_ARGS offsets, cell, frac, cs, n_src, g, tb, r0, r1, rec, status, grid, st
    switch (key) {
    case 1: return gather_launch<G, 1, 1>(FV_GATHER_ARGS);
    case 8: return gather_launch<G, 1, 8>(FV_GATHER_ARGS);
    case 12: return gather_launch<G, 1, 12>(FV_GATHER_ARGS);
    case 16: return gather_launch<G, 1, 16>(FV_GATHER_ARGS);
    case 101: return gather_launch<G, 4, 1>(FV_GATHER_ARGS);
    case 108:
        if constexpr (sizeof(G) == 4) return gather_launch<G, 4, 8>(FV_GATHER_ARGS);
        else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
#undef FV_GATHER_ARGS
}

template <class G>
cudaError_t launch_spread_tile(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                               const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                               cudaStream_t st)
{
    return gather_dispatch<G>(offsets, cell, frac, cs, n_src, g, tb, r0, r1, nullptr, nullptr, grid, st);
}

template <class G>
cudaError_t launch_spread_gather_rec(const int *offsets, const SrcRec<G> *rec, const cpx<G> *cs, const SliceGeom &g,
                                     const TimeBin &tb, double r0, double r1, int *status, cpx<G> *grid,
                                     cudaStream_t st)
{
    return gather_dispatch<G>(offsets, nullptr, nullptr, cs, 0, g, tb, r0, r1, rec, status, grid, st);
}

template cudaError_t launch_spread_gather_rec<float>(const int *, const SrcRec<float> *, const cpx<float> *,
                                                     const SliceGeom &, const TimeBin &, double, double, int *,
                                                     cpx<float> *, cudaStream_t);
template cudaError_t launch_spread_gather_rec<double>(const int *, const SrcRec<double> *, const cpx<double> *,
                                                      const SliceGeom &, const TimeBin &, double, double, int *,
                                                      cpx<double> *, cudaStream_t);

// Scatter form of the tiled spreading: a CTA owns a kScatX x kScatY tile with
// all z cells in shared memory (real and imaginary parts in separate planes,
// rows padded to kScatRS floats so that the lanes of a footprint fall in
// different banks); each warp takes one candidate source at a time, its lanes
// cover the source's (x, y) footprint inside the tile and loop over the z
// footprint, adding with shared-memory atomics; the tile is stored once.
constexpr int kScatX = 32, kScatY = 16, kScatRS = 40;

template <class G, int NP>
__global__ void __launch_bounds__(256, 4) k_spread_scatter(const int *__restrict__ offsets, const int *__restrict__ cell,
                                                        const G *__restrict__ frac, const cpx<G> *__restrict__ cs,
                                                        long n_src, SliceGeom g, TimeBin tb, double r0, double r1,
                                                        cpx<G> *__restrict__ grid)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.dim[0].nf1, ny = g.dim[1].nf1, nz = g.d == 3 ? g.dim[2].nf1 : 1;
    const int plane = nz * NP * kScatY * kScatRS;
    G *tre = reinterpret_cast<G *>(smem_raw), *tim = tre + plane;
    const int w = g.w;
    const int x0 = blockIdx.x * kScatX, y0 = blockIdx.y * kScatY;
    for (int i = threadIdx.x; i < 2 * plane; i += blockDim.x) tre[i] = (G)0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const double qx_lo = (x0 - nx / 2 - 0.5 * w) / r0, qx_hi = (x0 + kScatX - nx / 2 + 0.5 * w - 1) / r0;
    const double qy_lo = (y0 - ny / 2 - 0.5 * w) / r1, qy_hi = (y0 + kScatY - ny / 2 + 0.5 * w - 1) / r1;
    const int bx_lo = top_cell(qx_lo - 1.0, tb.nf1_top[0]) / tb.T[0];
    const int bx_hi = top_cell(qx_hi + 1.0, tb.nf1_top[0]) / tb.T[0];
    const int by_lo = top_cell(qy_lo - 1.0, tb.nf1_top[1]) / tb.T[1];
    const int by_hi = top_cell(qy_hi + 1.0, tb.nf1_top[1]) / tb.T[1];
    const G two_over_w = (G)2 / (G)w, beta = geom_beta<G>(g);
    __syncthreads();
    int k = 0;   // running candidate count across bin rows, dealt to warps round robin
    for (int by = by_lo; by <= by_hi; ++by) {
        const int i0 = offsets[by * tb.nbx + bx_lo], i1 = offsets[by * tb.nbx + bx_hi + 1];
        const int n = i1 - i0;
        int j = (warp - k % nwarps + nwarps) % nwarps;
        k += n;
        for (; j < n; j += nwarps) {
            const int i = i0 + j;
            const int cx = cell[i], cy = cell[n_src + i];
            if (cx + w <= x0 || cx >= x0 + kScatX || cy + w <= y0 || cy >= y0 + kScatY) continue;   // warp-uniform
            const int cz = g.d == 3 ? cell[2 * n_src + i] : 0;
            const G fx = frac[i], fy = frac[n_src + i];
            const G fz = g.d == 3 ? frac[2 * n_src + i] : (G)0;
            // z kernel values: lane jz < w computes one, every lane reads them by shuffle
            const G wz_mine = (g.d == 3 && lane < w) ? es_k<G>(two_over_w * (fz + (G)lane), beta) : (G)(lane == 0);
            cpx<G> c[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) c[p] = cs[(size_t)p * n_src + i];
            const int wzn = g.d == 3 ? w : 1;
            // every lane runs the same number of iterations: the shuffles below need the whole warp
            for (int pr0 = 0; pr0 < w * w; pr0 += 32) {
                const int pr = pr0 + lane;
                const int jy = pr / w, jx = pr - jy * w;
                const int lx = cx + jx - x0, ly = cy + jy - y0;
                const bool in = pr < w * w && lx >= 0 && lx < kScatX && ly >= 0 && ly < kScatY;
                const G wxy = in ? es_k<G>(two_over_w * (fx + (G)jx), beta) * es_k<G>(two_over_w * (fy + (G)jy), beta)
                                 : (G)0;
                const int cell_off = ly * kScatRS + lx;
                for (int jz = 0; jz < wzn; ++jz) {
                    const G wt = wxy * __shfl_sync(0xffffffffu, wz_mine, jz);
                    const int z = cz + jz;
                    if (in && z >= 0 && z < nz) {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const int o = (p * nz + z) * kScatY * kScatRS + cell_off;
                            atomicAdd(&tre[o], wt * c[p].x);
                            atomicAdd(&tim[o], wt * c[p].y);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const int tsz = NP * nz * kScatY * kScatX;
    for (int idx = threadIdx.x; idx < tsz; idx += blockDim.x) {
        const int lx = idx % kScatX;
        int rest = idx / kScatX;
        const int ly = rest % kScatY;
        rest /= kScatY;   // p * nz + z
        const int x = x0 + lx, y = y0 + ly;
        const int o = rest * kScatY * kScatRS + ly * kScatRS + lx;
        if (x < nx && y < ny) {
            const G sc = g.pre_x ? ((const G *)g.pre_x)[x] * ((const G *)g.pre_y)[y] : (G)1;
            grid[((size_t)rest * ny + y) * nx + x] = cmk<G>(tre[o] * sc, tim[o] * sc);
        }
    }
}

template <class G>
cudaError_t launch_spread_scatter(const int *offsets, const int *cell, const G *frac, const cpx<G> *cs, long n_src,
                                  const SliceGeom &g, const TimeBin &tb, double r0, double r1, cpx<G> *grid,
                                  cudaStream_t st)
{
    const int nz = g.d == 3 ? g.dim[2].nf1 : 1;
    const size_t smem = spread_scatter_smem(sizeof(G), g.n_pol, nz);
    if (smem > FV_SPREAD_SMEM_MAX || g.w > 32) return cudaErrorInvalidValue;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_spread_scatter<G, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, FV_SPREAD_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_spread_scatter<G, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, FV_SPREAD_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 blocks((g.dim[0].nf1 + kScatX - 1) / kScatX, (g.dim[1].nf1 + kScatY - 1) / kScatY);
    if (g.n_pol == 4)
        k_spread_scatter<G, 4><<<blocks, 256, smem, st>>>(offsets, cell, frac, cs, n_src, g, tb, r0, r1, grid);
    else
        k_spread_scatter<G, 1><<<blocks, 256, smem, st>>>(offsets, cell, frac, cs, n_src, g, tb, r0, r1, grid);
    return cudaGetLastError();
}

size_t spread_scatter_smem(int elem_bytes, int n_pol, int nz)
{
    return (size_t)2 * n_pol * nz * kScatY * kScatRS * elem_bytes;
}

template cudaError_t launch_spread_scatter<double>(const int *, const int *, const double *, const cpx<double> *, long,
                                                   const SliceGeom &, const TimeBin &, double, double,
                                                   cpx<double> *, cudaStream_t);
template cudaError_t launch_spread_scatter<float>(const int *, const int *, const float *, const cpx<float> *, long,
                                                  const SliceGeom &, const TimeBin &, double, double, cpx<float> *,
                                                  cudaStream_t);

template cudaError_t launch_prep<double>(const double *, const int *, const int *, long, const void *, int, int, int,
                                         const SliceGeom &, int *, double *, cpx<double> *, cudaStream_t);
template cudaError_t launch_prep<float>(const double *, const int *, const int *, long, const void *, int, int, int,
                                        const SliceGeom &, int *, float *, cpx<float> *, cudaStream_t);
template cudaError_t launch_prep_staged<double>(const double *, const int *, const int *, long, const void *, int,
                                                int, int, const SliceGeom &, SrcRec<double> *, cpx<double> *,
                                                cudaStream_t);
template cudaError_t launch_prep_staged<float>(const double *, const int *, const int *, long, const void *, int,
                                               int, int, const SliceGeom &, SrcRec<float> *, cpx<float> *,
                                               cudaStream_t);
template cudaError_t launch_spread_tile<double>(const int *, const int *, const double *, const cpx<double> *, long,
                                                const SliceGeom &, const TimeBin &, double, double, cpx<double> *,
                                                cudaStream_t);
template cudaError_t launch_spread_tile<float>(const int *, const int *, const float *, const cpx<float> *, long,
                                               const SliceGeom &, const TimeBin &, double, double, cpx<float> *,
                                               cudaStream_t);

}  // namespace fv
