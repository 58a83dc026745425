// Staged source records for the gather spreading (Section 2.2, step 1): the
// record layout that the prep kernel writes and the spreading kernel copies into
// shared memory in bulk, and the launchers of both.
#pragma once
#include "fv_internal.cuh"

namespace fv {

// Status bits a kernel may set in the plan's device status word.
#define FV_DEVICE_TIMEOUT 1

// ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on [-1, 1], zero outside (Section 2.2)
__device__ __forceinline__ double es_kernel_d(double z, double beta)
{
    double t = 1.0 - z * z;
    return t >= 0.0 ? exp(beta * (sqrt(t) - 1.0)) : 0.0;
}
__device__ __forceinline__ float es_kernel_f(float z, float beta)
{
    float t = 1.0f - z * z;
    return t >= 0.0f ? __expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}
template <class G> __device__ __forceinline__ G es_k(G z, G beta);
template <> __device__ __forceinline__ double es_k<double>(double z, double beta) { return es_kernel_d(z, beta); }
template <> __device__ __forceinline__ float es_k<float>(float z, float beta) { return es_kernel_f(z, beta); }

// Bulk asynchronous copies into shared memory, completion counted on an mbarrier (used by the gather
// kernel's record staging), and the bounded wait on a barrier phase.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init1(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// Wait for phase `parity` of *bar for at most about a second; false if the wait ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}

__device__ __forceinline__ int top_cell(double q, int nf1)
{
    double c = floor(q) + (double)(nf1 / 2);
    int ci = (int)fmax(0.0, fmin(c, (double)(nf1 - 1)));
    return ci;
}

// One source of one slice as the gather spreader reads it (16- or 32-byte records, copied in bulk):
// cell = cx | cy << 14 | cz << 28 (first footprint cell per axis; cx, cy < 16384, cz < 16) and the
// offsets frac = l0 - q of the grid coordinate split (Section 2.2).
template <class G> struct SrcRec;
template <> struct __align__(16) SrcRec<float> {
    unsigned cell;
    float fx, fy, fz;
};
template <> struct __align__(16) SrcRec<double> {
    unsigned cell, pad;
    double fx, fy, fz;
};

// One source of one slice as the ring gather (FP32 two-dimensional grids) reads it (80 bytes, copied in
// bulk): the packed first footprint cell (as in SrcRec) and the kernel values of its footprint columns and
// rows, phi((2/w)(f + j)) for j < w, zero for w <= j <= 8 (index 8 is always zero, so that a lookup
// clamped to 8 needs no test).
constexpr int kRingWmax = 8;
struct __align__(16) RingRec {
    unsigned cell;
    float wx[kRingWmax + 1], wy[kRingWmax + 1];
    unsigned pad;
};
static_assert(sizeof(RingRec) == 80, "ring records are 80 bytes (five 16-byte rows)");

// Complex strengths per source in the staged layout: n_pol values padded to a multiple of 16 bytes.
__host__ __device__ inline int staged_cs_stride(int elem, int n_pol)   // complex elements per source
{
    const int bytes = n_pol * 2 * elem;
    return ((bytes + 15) & ~15) / (2 * elem);
}

// The gather spreading (launch_spread_tile) reading staged records: each CTA's candidate chunks are copied
// into shared memory in bulk, double buffered.  Writes every cell of grid [n_pol][nz][ny][nx].
// status: device word; FV_DEVICE_TIMEOUT is or-ed in if a bounded wait on a copy ran out (the grid is
// then zero).  rec and cs must be readable 16 bytes past the last visible source.
template <class G>
cudaError_t launch_spread_gather_rec(const int *offsets, const SrcRec<G> *rec, const cpx<G> *cs, const SliceGeom &g,
                                     const TimeBin &tb, double r0, double r1, int *status, cpx<G> *grid,
                                     cudaStream_t st);

// Tiles of the ring gather: 32 x 16 cells, eight 8 x 8 blocks (one per consumer warp).  A tile with more
// than kRingPart candidates is split into parts of kRingPart candidates that different CTAs take; each
// part leaves its block sums in a slot and the last part of a tile to finish adds them up and stores the
// tile.  At most kRingSlotsMax parts per slice; tiles beyond them run whole.
constexpr int kRingTileX = 32, kRingTileY = 16, kRingBlocks = 8;
constexpr int kRingPart = 1024;
constexpr int kRingSlotsMax = 2048;
__host__ __device__ inline int ring_tiles(int nx, int ny)
{
    return ((nx + kRingTileX - 1) / kRingTileX) * ((ny + kRingTileY - 1) / kRingTileY);
}

// The work list of one ring-gather launch (device arrays of an execution workspace).
struct RingWork {
    int *hdr;          // [4]: ticket, parts of split tiles, unsplit tiles with candidates, tiles without
                       // (zero at the start of a slice: launch_prep_tc clears them)
    int4 *bins;        // [tiles]: bin rectangle (x0, x1, y0, y1) of a tile
    int *light;        // [tiles]: unsplit tiles with candidates from the front, tiles without from the back
    int4 *parts;       // [slots]: (tile, part, parts of the tile, the tile's first slot); tile -1: unused
    int *cnt;          // [tiles][kRingBlocks]: parts of a split tile finished, per block
    float4 *partial;   // [slots][kRingBlocks][n_pol][32 lanes]: a part's block sums
    int tiles, slots;
};

// The ring form of the same spreading for FP32 two-dimensional grids (n_pol 1 or 4, no height terms,
// w <= 8), reading ring records: a work-list kernel (bin rectangle and candidate count per tile, heavy
// tiles split into parts) and the gather itself: persistent CTAs, a producer warp streaming candidate
// chunks into a shared-memory ring, consumer warps summing 8 x 8 blocks with FP32 FMAs, or on the tensor
// cores when `tensor` is set.  cudaErrorInvalidValue for other slices or when the grid has more tiles
// than rw holds.  rw.hdr must be zero at launch (launch_prep_tc clears it).
cudaError_t launch_spread_ring(const int *offsets, const RingRec *rec, const cpx<float> *cs, const SliceGeom &g,
                               const TimeBin &tb, double r0, double r1, const RingWork &rw, int *status,
                               cpx<float> *grid, bool tensor, cudaStream_t st);

// Per slice: strengths with prephase and packed grid coordinates of the sorted sources, as staged
// records (the same arithmetic as launch_prep).
template <class G>
cudaError_t launch_prep_staged(const double *sdir, const int *sidx, const int *nv_ptr, long n_src,
                               const void *flux, int flux_fp64, int n_freq, int f, const SliceGeom &g,
                               SrcRec<G> *rec, cpx<G> *cs, cudaStream_t st);

// FP32 grids: the same, from the per-time records tc of launch_time_binning (no FP64 arithmetic); writes
// ring records when ring_rec is given (two-dimensional grids, w <= 8), else staged records when rec is
// given, else cell[3][n] / frac[3][n] / cs[n_pol][n].  tile_ctr (or nullptr): the four counters of the
// ring spreading's work list (RingWork::hdr), set to zero.  n_src must be > 0 when tile_ctr is given.
cudaError_t launch_prep_tc(const float4 *tc, const int *sidx, const int *nv_ptr, long n_src, const void *flux,
                           int flux_fp64, int n_freq, int f, const SliceGeom &g, int *cell, float *frac,
                           cpx<float> *cs, SrcRec<float> *rec, RingRec *ring_rec, int *tile_ctr, cudaStream_t st);

}  // namespace fv
