// Gather spreading of FP32 two-dimensional grids through a shared-memory ring (Section 2.2, step 1).
//
// A CTA works on a 32 x 16 tile at a time (4 x 2 blocks of 8 x 8 cells): eight consumer warps, one per
// block, and one producer warp.  A tile's candidates are the sources of the bins it maps to (one
// contiguous range of the sorted sources per bin row).  Sources are densest at the rim of the source
// disk, so a few tiles hold several times the mean count; a work-list kernel (k_ring_items) counts each
// tile's candidates and splits a tile with more than kRingPart of them into parts of kRingPart, so that
// the crowded tiles are summed by several CTAs at once.  CTAs are persistent (three per SM) and take
// work items (the parts first, then whole tiles) from an atomic ticket.  The producer copies an item's
// candidates into shared memory in chunks of 128 with bulk asynchronous copies into a three-stage ring
// (a full and an empty mbarrier per stage, every wait bounded) and runs ahead across item boundaries,
// so an item's first chunks are in flight while the consumers finish the previous one.  Each record
// already holds the source's kernel values (computed once per slice by the prep kernel), so a consumer
// warp only selects the chunk's candidates that overlap its block (ballot and prefix count, no shared
// atomics) and adds them; warps never wait for one another except through the ring.  A part leaves its
// block sums in a slot, and the last part of a tile to finish a block adds the other parts' sums to its
// own (a per-block counter, no waiting).  Every grid cell is stored once, with the x and y prescale of
// the FFT passes applied.
//
// The sum of a block's cells is
//     G(x, y) = sum_j c_j psi_y,j(y) psi_x,j(x)
// over its candidates j.  Two forms:
//  * FP32 FMAs (the default): lane (x, y) with x = lane & 7 holds rows y = lane >> 3 and y + 4 of its
//    column and adds c_j psi_x,j(x) psi_y,j(y) for every candidate that reaches those rows (one list per
//    half of the block), real and imaginary parts by one packed FP32 x 2 FMA, with FP32 accumulation;
//  * tensor cores (FV_SPREAD_TENSOR, an option): for an 8 x 8 block the sum is the matrix product D = A B
//    with A[(ri, y)][j] = Re / Im (c_j) psi_y,j(y) (16 x J) and B[j][x] = psi_x,j(x) (J x 8), taken eight
//    candidates at a time as m16n8k8 TF32 products with the three-term split
//    a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = tf32(a), a_lo = a - a_hi, of which the tensor core
//    reads the leading 11 bits): a relative error near 2^-21 per product.  Its operands are built in
//    registers, which is why it uses the warp-level mma.sync form: a block's A and B are sparse (a source
//    covers at most 7 of its 8 rows and columns, about a quarter on average) and change with every group
//    of eight candidates, so staging them through shared memory in the layouts tcgen05.mma reads would
//    cost more than the products.
#include "fv_staged.cuh"

#include <algorithm>
#include <climits>

namespace fv {

namespace {

constexpr int kRingConsumers = kRingBlocks;               // 4 x 2 blocks of 8 x 8
constexpr int kRingThreads = (kRingConsumers + 1) * 32;   // plus the producer warp
constexpr int kRingChunk = 128;
constexpr int kRingStages = 3;

__device__ __forceinline__ uint32_t to_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// D += A B, m16n8k8, A row-major (a0..a3), B column-major (b0, b1), FP32 accumulators d0..d3
__device__ __forceinline__ void mma_tf32(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mbar_init_n(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One selected candidate (list entry ent) into one half of a consumer lane's cells: a[p] += c_p psi_x psi_y
// with the lane's column and row given as ux = x + 16 and uy = y + 16 (the origin is stored + 16)
template <int NP>
__device__ __forceinline__ void ring_add(int ent, const RingRec *rec, const cpx<float> *cs, unsigned ux, unsigned uy,
                                         float2 (&a)[NP])
{
    constexpr int kCsw = (NP * 8 + 15) / 16 * 16 / 8;
    const int t = ent & 0xff;
    const RingRec &r = rec[t];
    const float wx = r.wx[min(ux - (((unsigned)ent >> 8) & 0xffu), (unsigned)kRingWmax)];
    const float wy = r.wy[min(uy - ((unsigned)ent >> 16), (unsigned)kRingWmax)];
    const float k = wx * wy;
    const float4 *c4 = reinterpret_cast<const float4 *>(cs + t * kCsw);
    float4 cv[NP > 1 ? 2 : 1];
#pragma unroll
    for (int q = 0; q < (NP > 1 ? 2 : 1); ++q) cv[q] = c4[q];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float4 u = cv[p >> 1];
        a[p] = __ffma2_rn(make_float2(k, k), (p & 1) ? make_float2(u.z, u.w) : make_float2(u.x, u.y), a[p]);
    }
}

}  // namespace

// The work list of one slice, one thread per tile: the tile's bin rectangle (the bins whose sources can
// reach it, through the top-grid mapping q = (x - nx / 2) / r with a margin of 1.25 top cells, which holds
// the FP32 rounding here and in the sources' coordinates many times over) and its candidate count; a tile
// with more than kRingPart candidates gets ceil(count / kRingPart) consecutive part slots (while slots are
// left), the others go to the unsplit list, those with candidates first.
__device__ __forceinline__ int ring_top_bin(float q, int nf1, int T)
{
    const float c = floorf(q) + (float)(nf1 / 2);
    return (int)fmaxf(0.0f, fminf(c, (float)(nf1 - 1))) / T;
}

__global__ void __launch_bounds__(64) k_ring_items(const int *__restrict__ offsets, TimeBin tb, int nx, int ny, int w,
                                                   float inv_r0, float inv_r1, int tiles_x, int n_tiles, RingWork rw)
{
    const int tile = blockIdx.x * 64 + threadIdx.x;
    if (tile >= n_tiles) return;
    const int x0 = (tile % tiles_x) * kRingTileX, y0 = (tile / tiles_x) * kRingTileY;
    const float hw = 0.5f * (float)w;
    const int4 bn = make_int4(ring_top_bin(((float)(x0 - nx / 2) - hw) * inv_r0 - 1.25f, tb.nf1_top[0], tb.T[0]),
                              ring_top_bin(((float)(x0 + kRingTileX - 1 - nx / 2) + hw) * inv_r0 + 1.25f, tb.nf1_top[0], tb.T[0]),
                              ring_top_bin(((float)(y0 - ny / 2) - hw) * inv_r1 - 1.25f, tb.nf1_top[1], tb.T[1]),
                              ring_top_bin(((float)(y0 + kRingTileY - 1 - ny / 2) + hw) * inv_r1 + 1.25f, tb.nf1_top[1], tb.T[1]));
    rw.bins[tile] = bn;
    long total = 0;
#pragma unroll 4
    for (int r = bn.z; r <= bn.w; ++r) total += offsets[r * tb.nbx + bn.y + 1] - offsets[r * tb.nbx + bn.x];
    if (total == 0) {
        rw.light[n_tiles - 1 - atomicAdd(&rw.hdr[3], 1)] = tile;
        return;
    }
    if (total > kRingPart) {
        // consecutive slots for the parts; where they run past the end, the slots that were taken are
        // marked empty (tile -1) and the tile runs whole
        const int np = (int)((total + kRingPart - 1) / kRingPart);
        const int first = atomicAdd(&rw.hdr[1], np);
        if (first + np <= rw.slots) {
            for (int k = 0; k < np; ++k) rw.parts[first + k] = make_int4(tile, k, np, first);
            for (int b = 0; b < kRingBlocks; ++b) rw.cnt[tile * kRingBlocks + b] = 0;
            return;
        }
        for (int k = first; k < rw.slots; ++k) rw.parts[k] = make_int4(-1, 0, 1, 0);
    }
    rw.light[atomicAdd(&rw.hdr[2], 1)] = tile;     // unsplit
}

template <int NP, bool TC>
__global__ void __launch_bounds__(kRingThreads, 3) k_spread_ring(const int *__restrict__ offsets,
                                                            const RingRec *__restrict__ rec,
                                                            const cpx<float> *__restrict__ cs, SliceGeom g, TimeBin tb,
                                                            int tiles_x, int n_tiles, RingWork rw,
                                                            int *__restrict__ status, cpx<float> *__restrict__ grid)
{
    constexpr int kCsw = (NP * 8 + 15) / 16 * 16 / 8;           // staged strengths per source (16-byte rows)
    __shared__ __align__(16) RingRec s_rec[kRingStages][kRingChunk];
    __shared__ __align__(16) cpx<float> s_cs[kRingStages][kRingChunk * kCsw];
    __shared__ __align__(8) uint64_t s_full[kRingStages], s_empty[kRingStages];
    // per stage: candidates of a chunk, or -1 for a work-item boundary whose next item is tile s_tile,
    // part (bits 0-15) of s_part >> 16 parts, the tile's first part slot s_slot
    __shared__ int s_n[kRingStages], s_tile[kRingStages], s_part[kRingStages], s_slot[kRingStages];
    // a warp's selected candidates: t (bits 0-7) and the footprint origin relative to the block + 16 in x
    // (bits 8-15) and y (bits 16-23); the FP32 form keeps the candidates that reach the block's rows 0-3
    // from the front and those that reach rows 4-7 from the back (a candidate may be in both)
    __shared__ int s_sel[kRingConsumers][TC ? kRingChunk : 2 * kRingChunk];
    __shared__ int s_row0[32], s_pre[32];                         // the producer's rows table
    __shared__ int s_abort;
    const int nx = g.dim[0].nf1, ny = g.dim[1].nf1;
    const int w = g.w;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kRingStages; ++b) {
            mbar_init_n(&s_full[b], 1);
            mbar_init_n(&s_empty[b], kRingConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    volatile int *abort_flag = &s_abort;

    // Work items (a tile, or a part of a split tile) are handed out by an atomic ticket (rw.hdr[0], zeroed
    // by the prep kernel before this launch); the producer runs ahead across item boundaries, so the next
    // item's first chunks are in flight while the consumers finish the current one.
    if (warp == kRingConsumers) {
        // ---------------- producer warp: work items, rows tables and bulk copies of the candidate chunks
        int kc = 0;              // stages filled
        unsigned ephase = 0u;    // bit b: parity of the next completion of stage b's empty barrier
        int ok = 1;
        // the work list (complete: the work-list kernel ran before this launch): parts of split tiles, then
        // unsplit tiles with candidates, then tiles without
        const int n_split = min(rw.hdr[1], rw.slots), n_light = rw.hdr[2], n_empty = rw.hdr[3];
        // lane 0: wait until stage kc % kRingStages is free (its previous use consumed); false if that ran out
        auto acquire = [&](int b) -> bool {
            if (kc < kRingStages) return true;
            const bool got = mbar_wait(&s_empty[b], (ephase >> b) & 1u);
            ephase ^= 1u << b;
            return got && !*abort_flag;
        };
        // lane 0: take the next work item (tile, part, parts, first slot; tile n_tiles when none is left)
        // and announce it with a boundary stage
        auto next_item = [&]() -> int4 {
            int t = atomicAdd(&rw.hdr[0], 1);
            // slots marked empty are passed over (at most n_split of them)
            while (t < n_split && rw.parts[t].x < 0) t = atomicAdd(&rw.hdr[0], 1);
            int4 it = make_int4(n_tiles, 0, 1, 0);
            if (t < n_split) it = rw.parts[t];
            else if (t < n_split + n_light) it.x = rw.light[t - n_split];
            else if (t < n_split + n_light + n_empty) it.x = rw.light[n_tiles - 1 - (t - n_split - n_light)];
            const int b = kc % kRingStages;
            if (!acquire(b)) {
                ok = 0;
                it.x = n_tiles;
                return it;
            }
            s_n[b] = -1;
            s_tile[b] = it.x;
            s_part[b] = it.y | (it.z << 16);
            s_slot[b] = it.w;
            mbar_arrive(&s_full[b]);
            ++kc;
            return it;
        };
        int4 item = make_int4(n_tiles, 0, 1, 0);
        if (lane == 0) item = next_item();
        auto share = [&]() {
            item.x = __shfl_sync(0xffffffffu, item.x, 0);
            item.y = __shfl_sync(0xffffffffu, item.y, 0);
            item.z = __shfl_sync(0xffffffffu, item.z, 0);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            kc = __shfl_sync(0xffffffffu, kc, 0);
            ephase = __shfl_sync(0xffffffffu, ephase, 0);
        };
        share();
        while (item.x < n_tiles && ok) {
            const int4 bn = rw.bins[item.x];       // bin rectangle: x0, x1, y0, y1
            // the part's range [plo, phi) of the tile's candidates in row order (all of an unsplit tile's)
            const long plo = (long)item.y * kRingPart, phi = item.z > 1 ? plo + kRingPart : LONG_MAX;
            long gbase = 0;                          // candidates in the bin rows before this group
            for (int r0w = bn.z; r0w <= bn.w && ok && gbase < phi; r0w += 32) {
                const int nrows = min(32, bn.w - r0w + 1);
                int start = 0, len = 0;
                if (lane < nrows) {
                    const int row = (r0w + lane) * tb.nbx;
                    start = offsets[row + bn.x];
                    len = offsets[row + bn.y + 1] - start;
                }
                int incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                s_row0[lane] = start;
                s_pre[lane] = incl - len;
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                // this part's candidates among the group's
                const int a0 = (int)max(plo - gbase, 0L), a1 = (int)min(phi - gbase, (long)total);
                __syncwarp();
                if (lane == 0) {
                    for (int base = a0; base < a1; base += kRingChunk) {
                        const int b = kc % kRingStages;
                        if (!acquire(b)) {
                            ok = 0;
                            break;
                        }
                        const int n = min(kRingChunk, a1 - base);
                        s_n[b] = n;
                        mbar_expect(&s_full[b], (unsigned)n * (unsigned)(sizeof(RingRec) + kCsw * sizeof(cpx<float>)));
                        for (int r = 0; r < nrows; ++r) {
                            const int rlen = (r + 1 < nrows ? s_pre[r + 1] : total) - s_pre[r];
                            const int a = max(base, s_pre[r]), e = min(base + n, s_pre[r] + rlen);
                            if (a >= e) continue;
                            const int i0 = s_row0[r] + (a - s_pre[r]), m = e - a;
                            bulk_g2s(&s_rec[b][a - base], rec + i0, (unsigned)(m * sizeof(RingRec)), &s_full[b]);
                            bulk_g2s(&s_cs[b][(a - base) * kCsw], cs + (size_t)i0 * kCsw,
                                     (unsigned)(m * kCsw * sizeof(cpx<float>)), &s_full[b]);
                        }
                        ++kc;
                    }
                }
                gbase += total;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                kc = __shfl_sync(0xffffffffu, kc, 0);
                ephase = __shfl_sync(0xffffffffu, ephase, 0);
                __syncwarp();    // lane 0 is done with the rows table before the next group rewrites it
            }
            if (!ok) break;
            if (lane == 0) item = next_item();
            share();
        }
        if (lane == 0 && !ok) {
            // a wait ran out: tell the consumers, record it, and wait (bounded) for the copies in flight
            *abort_flag = 1;
            atomicOr(status, FV_DEVICE_TIMEOUT);
            for (int k = max(0, kc - kRingStages); k < kc; ++k)
                mbar_wait(&s_full[k % kRingStages], (unsigned)(k / kRingStages) & 1u);
        }
        return;
    }

    // ---------------- consumer warps: one 8 x 8 block of each tile
    const int gq = lane >> 2, tq = lane & 3;                             // fragment group, k index
    unsigned fphase = 0u;    // bit b: parity of the next completion of stage b's full barrier
    int tile = -1;           // none yet
    int part = 0, nparts = 1, slot0 = 0;    // the current item's part of its tile, and the tile's first slot
    int bx0 = 0, by0 = 0;    // the block's first cell
    float d[NP][4];         // tensor form: the D fragments
    float2 acc[2][NP];      // FP32 form: rows y and y + 4 of the lane's column, (Re, Im) per product
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int k = 0; k < 4; ++k) d[p][k] = 0.0f;
        acc[0][p] = acc[1][p] = make_float2(0.0f, 0.0f);
    }
    for (int kc = 0;; ++kc) {
        const int b = kc % kRingStages;
        // the lanes decide together: a wait that ran out on any lane, or an abort, ends the warp's work
        const bool got = __all_sync(0xffffffffu, mbar_wait(&s_full[b], (fphase >> b) & 1u));
        const int aborted = __shfl_sync(0xffffffffu, *abort_flag, 0);
        fphase ^= 1u << b;
        if (!got || aborted) {
            if (lane == 0 && !got) {
                *abort_flag = 1;
                atomicOr(status, FV_DEVICE_TIMEOUT);
            }
            break;
        }
        const int n = s_n[b], next = s_tile[b], next_part = s_part[b], next_slot = s_slot[b];
        if (n > 0) {
            // the chunk's candidates whose footprint overlaps this block, in order
            int L = 0, L4 = 0;
            for (int c0 = 0; c0 < n; c0 += 32) {
                const int t = c0 + lane;
                bool hit = false, top = false;
                int ent = 0;
                if (t < n) {
                    const unsigned cell = s_rec[b][t].cell;
                    const int cx = (int)(cell & 0x3fffu) - bx0, cy = (int)((cell >> 14) & 0x3fffu) - by0;
                    hit = cx <= 7 && cx + w > 0 && cy <= 7 && cy + w > 0;    // then -15 < cx, cy <= 7
                    ent = t | ((cx + 16) << 8) | ((cy + 16) << 16);
                    if (!TC) {
                        top = hit && cy + w > 4;       // reaches rows 4-7
                        hit = hit && cy <= 3;          // reaches rows 0-3
                    }
                }
                const unsigned below = (1u << lane) - 1u;
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) s_sel[warp][L + __popc(m & below)] = ent;
                L += __popc(m);
                if (!TC) {
                    const unsigned m4 = __ballot_sync(0xffffffffu, top);
                    if (top) s_sel[warp][2 * kRingChunk - 1 - (L4 + __popc(m4 & below))] = ent;
                    L4 += __popc(m4);
                }
            }
            __syncwarp();
            if (!TC) {
                // FP32 FMAs: lane (x = lane & 7, rows y = lane >> 3 and y + 4) adds c psi_x(x) psi_y(y) of every
                // selected candidate into its cells, the real and imaginary parts by one packed FP32 x 2 FMA.
                // A candidate is taken once per half of the block it reaches; lanes outside its footprint
                // read the zero kernel value at index 8.
                const unsigned ux = (unsigned)((lane & 7) + 16), uy = (unsigned)((lane >> 3) + 16);
#pragma unroll 4
                for (int e = 0; e < L; ++e)
                    ring_add<NP>(s_sel[warp][e], s_rec[b], s_cs[b], ux, uy, acc[0]);
#pragma unroll 4
                for (int e = 0; e < L4; ++e)
                    ring_add<NP>(s_sel[warp][2 * kRingChunk - 1 - e], s_rec[b], s_cs[b], ux, uy + 4u, acc[1]);
            }
            // eight candidates per product: this lane supplies k = tq (h = 0) and k = tq + 4 (h = 1)
            for (int e = 0; TC && e < L; e += 8) {
                uint32_t bh[2], bl[2];
                float wy[2];
                float4 cv[2][NP > 1 ? 2 : 1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = e + tq + 4 * h;
                    float wx = 0.0f;
                    wy[h] = 0.0f;
                    int t = 0;
                    if (k < L) {
                        const int ent = s_sel[warp][k];
                        t = ent & 0xff;
                        const RingRec &r = s_rec[b][t];
                        const unsigned dx = (unsigned)(gq + 16 - ((ent >> 8) & 0xff));
                        const unsigned dy = (unsigned)(gq + 16 - (ent >> 16));
                        if (dx < (unsigned)kRingWmax) wx = r.wx[dx];      // zero past w
                        if (dy < (unsigned)kRingWmax) wy[h] = r.wy[dy];
                    }
                    // B: hi = tf32(wx); lo = the remainder, whose low bits the tensor core ignores
                    bh[h] = to_tf32(wx);
                    bl[h] = __float_as_uint(wx - __uint_as_float(bh[h]));
                    const float4 *c4 = reinterpret_cast<const float4 *>(&s_cs[b][t * kCsw]);
#pragma unroll
                    for (int q = 0; q < (NP > 1 ? 2 : 1); ++q) cv[h][q] = c4[q];
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float4 u0 = cv[0][p >> 1], u1 = cv[1][p >> 1];
                    const float re0 = (p & 1) ? u0.z : u0.x, im0 = (p & 1) ? u0.w : u0.y;
                    const float re1 = (p & 1) ? u1.z : u1.x, im1 = (p & 1) ? u1.w : u1.y;
                    // a0 = (row gq, k tq): Re, a1 = (gq + 8, tq): Im, a2 = (gq, tq + 4): Re, a3 = (gq + 8, tq + 4): Im
                    const float a0 = re0 * wy[0], a1 = im0 * wy[0], a2 = re1 * wy[1], a3 = im1 * wy[1];
                    const uint32_t h0 = to_tf32(a0), h1 = to_tf32(a1), h2 = to_tf32(a2), h3 = to_tf32(a3);
                    mma_tf32(d[p], __float_as_uint(a0 - __uint_as_float(h0)), __float_as_uint(a1 - __uint_as_float(h1)),
                             __float_as_uint(a2 - __uint_as_float(h2)), __float_as_uint(a3 - __uint_as_float(h3)),
                             bh[0], bh[1]);
                    mma_tf32(d[p], h0, h1, h2, h3, bl[0], bl[1]);
                    mma_tf32(d[p], h0, h1, h2, h3, bh[0], bh[1]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[b]);      // after the stage was read
        if (n < 0) {
            bool store = tile >= 0;
            if (store && nparts > 1) {
                // a part of a split tile: its block sums go to the part's slot, and the last of the tile's
                // parts to finish this block adds the others' to its own and stores the block
                float4 *mine = rw.partial + ((size_t)(slot0 + part) * kRingBlocks + warp) * NP * 32 + lane;
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    mine[p * 32] = TC ? make_float4(d[p][0], d[p][1], d[p][2], d[p][3])
                                      : make_float4(acc[0][p].x, acc[0][p].y, acc[1][p].x, acc[1][p].y);
                __threadfence();
                __syncwarp();
                int done = 0;
                if (lane == 0) done = atomicAdd(&rw.cnt[tile * kRingBlocks + warp], 1);
                store = __shfl_sync(0xffffffffu, done, 0) == nparts - 1;
                if (store) {
                    __threadfence();
                    for (int j = 0; j < nparts; ++j) {
                        if (j == part) continue;
                        const float4 *o = rw.partial + ((size_t)(slot0 + j) * kRingBlocks + warp) * NP * 32 + lane;
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const float4 v = __ldcg(o + p * 32);
                            if (TC) {
                                d[p][0] += v.x;
                                d[p][1] += v.y;
                                d[p][2] += v.z;
                                d[p][3] += v.w;
                            } else {
                                acc[0][p].x += v.x;
                                acc[0][p].y += v.y;
                                acc[1][p].x += v.z;
                                acc[1][p].y += v.w;
                            }
                        }
                    }
                }
            }
            if (store && !TC) {
                // this lane's cells: (bx0 + lane & 7, by0 + lane >> 3) in acc[0], four rows down in acc[1]
                const int x = bx0 + (lane & 7);
                const float *px = (const float *)g.pre_x, *py = (const float *)g.pre_y;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int y = by0 + (lane >> 3) + 4 * c;
                    if (x < nx && y < ny) {
                        const float sc = (py ? py[y] : 1.0f) * (px ? px[x] : 1.0f);
#pragma unroll
                        for (int p = 0; p < NP; ++p)
                            grid[((size_t)p * ny + y) * nx + x] = cmk<float>(acc[c][p].x * sc, acc[c][p].y * sc);
                    }
                }
            }
            if (store && TC) {
                // D fragment of product p: d0 = Re (row gq, column 2 tq), d1 = Re (gq, 2 tq + 1),
                // d2 = Im (gq, 2 tq), d3 = Im (gq, 2 tq + 1); rows are y and columns x of the block
                const int gy = by0 + gq, gx = bx0 + 2 * tq;
                if (gy < ny) {
                    const float *px = (const float *)g.pre_x, *py = (const float *)g.pre_y;
                    const float sy = py ? py[gy] : 1.0f;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int x = gx + c;
                        if (x < nx) {
                            const float sc = sy * (px ? px[x] : 1.0f);
#pragma unroll
                            for (int p = 0; p < NP; ++p)
                                grid[((size_t)p * ny + gy) * nx + x] = cmk<float>(d[p][c] * sc, d[p][2 + c] * sc);
                        }
                    }
                }
            }
            if (tile >= 0) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) d[p][k] = 0.0f;
                    acc[0][p] = acc[1][p] = make_float2(0.0f, 0.0f);
                }
            }
            tile = next;
            part = next_part & 0xffff;
            nparts = next_part >> 16;
            slot0 = next_slot;
            if (tile >= n_tiles) break;
            bx0 = (tile % tiles_x) * kRingTileX + (warp & 3) * 8;
            by0 = (tile / tiles_x) * kRingTileY + (warp >> 2) * 8;
        }
    }
}

// The ring gather for an FP32 two-dimensional slice (n_pol 1 or 4, w <= 8) from ring records (launch_prep_tc);
// tensor: the block sums on the tensor cores.  Writes every cell of grid [n_pol][ny][nx].
cudaError_t launch_spread_ring(const int *offsets, const RingRec *rec, const cpx<float> *cs, const SliceGeom &g,
                               const TimeBin &tb, double r0, double r1, const RingWork &rw, int *status,
                               cpx<float> *grid, bool tensor, cudaStream_t st)
{
    if (g.d != 2 || g.K != 0 || g.w > kRingWmax || (g.n_pol != 1 && g.n_pol != 4)) return cudaErrorInvalidValue;
    const int tiles_x = (g.dim[0].nf1 + kRingTileX - 1) / kRingTileX;
    const int n_tiles = ring_tiles(g.dim[0].nf1, g.dim[1].nf1);
    if (!rw.hdr || n_tiles > rw.tiles || rw.slots < 0) return cudaErrorInvalidValue;
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev]) {
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    k_ring_items<<<(n_tiles + 63) / 64, 64, 0, st>>>(offsets, tb, g.dim[0].nf1, g.dim[1].nf1, g.w, (float)(1.0 / r0),
                                                     (float)(1.0 / r1), tiles_x, n_tiles, rw);
    // persistent: three CTAs per SM (the register and shared-memory budget), each taking work items by ticket
    const unsigned blocks = (unsigned)std::max(1, std::min(n_tiles + rw.slots, 3 * sms[dev]));
#define FV_RING_ARGS offsets, rec, cs, g, tb, tiles_x, n_tiles, rw, status, grid
    if (g.n_pol == 4) {
        if (tensor) k_spread_ring<4, true><<<blocks, kRingThreads, 0, st>>>(FV_RING_ARGS);
        else k_spread_ring<4, false><<<blocks, kRingThreads, 0, st>>>(FV_RING_ARGS);
    } else {
        if (tensor) k_spread_ring<1, true><<<blocks, kRingThreads, 0, st>>>(FV_RING_ARGS);
        else k_spread_ring<1, false><<<blocks, kRingThreads, 0, st>>>(FV_RING_ARGS);
    }
#undef FV_RING_ARGS
    return cudaGetLastError();
}

}  // namespace fv
