// Gather spreading of FP32 two-dimensional grids through a shared-memory ring (Section 2.2, step 1).
//
// A CTA owns a 32 x 16 tile at a time (4 x 2 blocks of 8 x 8 cells): eight consumer warps, one per
// block, and one producer warp.  CTAs are persistent (three per SM) and take tiles from an atomic
// ticket.  A tile's candidates are the sources of the bins it maps to (one contiguous range of the sorted
// sources per bin row); the producer copies them into shared memory in chunks of 128 with bulk
// asynchronous copies into a three-stage ring (a full and an empty mbarrier per stage, every wait
// bounded) and runs ahead across tile boundaries, so a tile's first chunks are in flight while the
// consumers finish the previous one.  Each record already holds the source's kernel values (computed
// once per slice by the prep kernel), so a consumer warp only selects the chunk's candidates that
// overlap its block (ballot and prefix count, no shared atomics) and adds them; warps never wait for one
// another except through the ring.  Every grid cell is stored once, with the x and y prescale of the FFT
// passes applied.
//
// The sum of a block's cells is
//     G(x, y) = sum_j c_j psi_y,j(y) psi_x,j(x)
// over its candidates j.  Two forms:
//  * FP32 FMAs (the default): lane (x, y) with x = lane & 7 holds rows y = lane >> 3 and y + 4 of its
//    column and adds c_j psi_x,j(x) psi_y,j(y) for every candidate, in FP32 with FP32 accumulation;
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

namespace fv {

namespace {

constexpr int kRingConsumers = 8;                       // 4 x 2 blocks of 8 x 8
constexpr int kRingThreads = (kRingConsumers + 1) * 32;   // plus the producer warp
constexpr int kRingTileX = 32, kRingTileY = 16;
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

}  // namespace

template <int NP, bool TC>
__global__ void __launch_bounds__(kRingThreads, 3) k_spread_ring(const int *__restrict__ offsets,
                                                            const RingRec *__restrict__ rec,
                                                            const cpx<float> *__restrict__ cs, SliceGeom g, TimeBin tb,
                                                            double r0, double r1, int tiles_x, int n_tiles,
                                                            int *__restrict__ tile_ctr, int *__restrict__ status,
                                                            cpx<float> *__restrict__ grid)
{
    constexpr int kCsw = (NP * 8 + 15) / 16 * 16 / 8;           // staged strengths per source (16-byte rows)
    __shared__ __align__(16) RingRec s_rec[kRingStages][kRingChunk];
    __shared__ __align__(16) cpx<float> s_cs[kRingStages][kRingChunk * kCsw];
    __shared__ __align__(8) uint64_t s_full[kRingStages], s_empty[kRingStages];
    // per stage: candidates of a chunk, or -1 for a tile boundary whose next tile is s_tile
    __shared__ int s_n[kRingStages], s_tile[kRingStages];
    // a warp's selected candidates: t (bits 0-7) and the footprint origin relative to the block + 16 in x
    // (bits 8-15) and y (bits 16-23)
    __shared__ int s_sel[kRingConsumers][kRingChunk];
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

    // Tiles are handed out by an atomic ticket (tile_ctr, zeroed by the prep kernel before this launch);
    // the producer runs ahead across tile boundaries, so the next tile's first chunks are in flight while
    // the consumers finish the current one.
    if (warp == kRingConsumers) {
        // ---------------- producer warp: tiles, rows tables and bulk copies of the candidate chunks
        int kc = 0;              // stages filled
        unsigned ephase = 0u;    // bit b: parity of the next completion of stage b's empty barrier
        int ok = 1;
        // lane 0: wait until stage kc % kRingStages is free (its previous use consumed); false if that ran out
        auto acquire = [&](int b) -> bool {
            if (kc < kRingStages) return true;
            const bool got = mbar_wait(&s_empty[b], (ephase >> b) & 1u);
            ephase ^= 1u << b;
            return got && !*abort_flag;
        };
        // lane 0: take the next tile and announce it with a boundary stage
        auto next_tile = [&]() -> int {
            const int t = atomicAdd(tile_ctr, 1);
            const int b = kc % kRingStages;
            if (!acquire(b)) {
                ok = 0;
                return n_tiles;
            }
            s_n[b] = -1;
            s_tile[b] = t;
            mbar_arrive(&s_full[b]);
            ++kc;
            return t;
        };
        int tile = lane == 0 ? next_tile() : 0;
        tile = __shfl_sync(0xffffffffu, tile, 0);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        kc = __shfl_sync(0xffffffffu, kc, 0);
        while (tile < n_tiles && ok) {
            const int x0 = (tile % tiles_x) * kRingTileX, y0 = (tile / tiles_x) * kRingTileY;
            int bins[4] = {0, 0, 0, 0};
            if (lane == 0) {
                // the bin rectangle of the tile (one-cell margin through the top-grid mapping), in FP64
                const double qx_lo = (x0 - nx / 2 - 0.5 * w) / r0;
                const double qx_hi = (x0 + kRingTileX - nx / 2 + 0.5 * w - 1) / r0;
                const double qy_lo = (y0 - ny / 2 - 0.5 * w) / r1;
                const double qy_hi = (y0 + kRingTileY - ny / 2 + 0.5 * w - 1) / r1;
                bins[0] = top_cell(qx_lo - 1.0, tb.nf1_top[0]) / tb.T[0];
                bins[1] = top_cell(qx_hi + 1.0, tb.nf1_top[0]) / tb.T[0];
                bins[2] = top_cell(qy_lo - 1.0, tb.nf1_top[1]) / tb.T[1];
                bins[3] = top_cell(qy_hi + 1.0, tb.nf1_top[1]) / tb.T[1];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) bins[k] = __shfl_sync(0xffffffffu, bins[k], 0);
            for (int r0w = bins[2]; r0w <= bins[3] && ok; r0w += 32) {
                const int nrows = min(32, bins[3] - r0w + 1);
                int start = 0, len = 0;
                if (lane < nrows) {
                    const int row = (r0w + lane) * tb.nbx;
                    start = offsets[row + bins[0]];
                    len = offsets[row + bins[1] + 1] - start;
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
                __syncwarp();
                if (lane == 0) {
                    for (int base = 0; base < total; base += kRingChunk) {
                        const int b = kc % kRingStages;
                        if (!acquire(b)) {
                            ok = 0;
                            break;
                        }
                        const int n = min(kRingChunk, total - base);
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
                ok = __shfl_sync(0xffffffffu, ok, 0);
                kc = __shfl_sync(0xffffffffu, kc, 0);
                ephase = __shfl_sync(0xffffffffu, ephase, 0);
                __syncwarp();    // lane 0 is done with the rows table before the next group rewrites it
            }
            if (!ok) break;
            tile = lane == 0 ? next_tile() : 0;
            tile = __shfl_sync(0xffffffffu, tile, 0);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            kc = __shfl_sync(0xffffffffu, kc, 0);
            ephase = __shfl_sync(0xffffffffu, ephase, 0);
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
    int bx0 = 0, by0 = 0;    // the block's first cell
    float d[NP][4];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int k = 0; k < 4; ++k) d[p][k] = 0.0f;
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
        const int n = s_n[b], next = s_tile[b];
        if (n > 0) {
            // the chunk's candidates whose footprint overlaps this block, in order
            int L = 0;
            for (int c0 = 0; c0 < n; c0 += 32) {
                const int t = c0 + lane;
                bool hit = false;
                int ent = 0;
                if (t < n) {
                    const unsigned cell = s_rec[b][t].cell;
                    const int cx = (int)(cell & 0x3fffu) - bx0, cy = (int)((cell >> 14) & 0x3fffu) - by0;
                    hit = cx <= 7 && cx + w > 0 && cy <= 7 && cy + w > 0;    // then -15 < cx, cy <= 7
                    ent = t | ((cx + 16) << 8) | ((cy + 16) << 16);
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) s_sel[warp][L + __popc(m & ((1u << lane) - 1u))] = ent;
                L += __popc(m);
            }
            __syncwarp();
            if (!TC) {
                // FP32 FMAs: lane (x = lane & 7, rows lane >> 3 and + 4) adds every selected candidate's
                // c psi_x(x) psi_y(y) into its two cells; out-of-footprint lanes add zero weights
                const int lx = lane & 7, ly = lane >> 3;
#pragma unroll 2
                for (int e = 0; e < L; ++e) {
                    const int ent = s_sel[warp][e];
                    const int t = ent & 0xff;
                    const RingRec &r = s_rec[b][t];
                    const unsigned dx = (unsigned)(lx + 16 - ((ent >> 8) & 0xff));
                    const unsigned dy0 = (unsigned)(ly + 16 - (ent >> 16)), dy1 = dy0 + 4u;
                    const float wx = dx < (unsigned)kRingWmax ? r.wx[dx] : 0.0f;
                    const float wy0 = dy0 < (unsigned)kRingWmax ? r.wy[dy0] : 0.0f;
                    const float wy1 = dy1 < (unsigned)kRingWmax ? r.wy[dy1] : 0.0f;
                    const float4 *c4 = reinterpret_cast<const float4 *>(&s_cs[b][t * kCsw]);
                    float4 cv[NP > 1 ? 2 : 1];
#pragma unroll
                    for (int q = 0; q < (NP > 1 ? 2 : 1); ++q) cv[q] = c4[q];
                    const float k0 = wx * wy0, k1 = wx * wy1;     // the two cells' kernel weights
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const float4 u = cv[p >> 1];
                        const float cr = (p & 1) ? u.z : u.x, ci = (p & 1) ? u.w : u.y;
                        d[p][0] = fmaf(k0, cr, d[p][0]);
                        d[p][1] = fmaf(k0, ci, d[p][1]);
                        d[p][2] = fmaf(k1, cr, d[p][2]);
                        d[p][3] = fmaf(k1, ci, d[p][3]);
                    }
                }
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
            if (tile >= 0 && !TC) {
                // this lane's cells: (bx0 + lane & 7, by0 + lane >> 3) in d[p][0..1], four rows down in d[p][2..3]
                const int x = bx0 + (lane & 7);
                const float *px = (const float *)g.pre_x, *py = (const float *)g.pre_y;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int y = by0 + (lane >> 3) + 4 * c;
                    if (x < nx && y < ny) {
                        const float sc = (py ? py[y] : 1.0f) * (px ? px[x] : 1.0f);
#pragma unroll
                        for (int p = 0; p < NP; ++p)
                            grid[((size_t)p * ny + y) * nx + x] = cmk<float>(d[p][2 * c] * sc, d[p][2 * c + 1] * sc);
                    }
                }
            }
            if (tile >= 0 && TC) {
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
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int k = 0; k < 4; ++k) d[p][k] = 0.0f;
            }
            tile = next;
            if (tile >= n_tiles) break;
            bx0 = (tile % tiles_x) * kRingTileX + (warp & 3) * 8;
            by0 = (tile / tiles_x) * kRingTileY + (warp >> 2) * 8;
        }
    }
}

// The ring gather for an FP32 two-dimensional slice (n_pol 1 or 4, w <= 8) from ring records (launch_prep_tc);
// tensor: the block sums on the tensor cores.  Writes every cell of grid [n_pol][ny][nx].
cudaError_t launch_spread_ring(const int *offsets, const RingRec *rec, const cpx<float> *cs, const SliceGeom &g,
                               const TimeBin &tb, double r0, double r1, int *tile_ctr, int *status, cpx<float> *grid,
                               bool tensor, cudaStream_t st)
{
    if (g.d != 2 || g.K != 0 || g.w > kRingWmax || (g.n_pol != 1 && g.n_pol != 4)) return cudaErrorInvalidValue;
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev]) {
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    // persistent: three CTAs per SM (the register and shared-memory budget), each taking tiles by ticket
    const int tiles_x = (g.dim[0].nf1 + kRingTileX - 1) / kRingTileX;
    const int n_tiles = tiles_x * ((g.dim[1].nf1 + kRingTileY - 1) / kRingTileY);
    const unsigned blocks = (unsigned)std::max(1, std::min(n_tiles, 3 * sms[dev]));
#define FV_RING_ARGS offsets, rec, cs, g, tb, r0, r1, tiles_x, n_tiles, tile_ctr, status, grid
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
