// fv_execute_static: fv_execute for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at the point where
// they want visibilities: a host framework that owns the whole device memory
// through its own allocator (a caching pool that already holds the free HBM,
// so a foreign cudaMalloc fails or fragments it), a serving loop that admits
// work against a fixed HBM budget and must not grow its footprint while it
// runs, or a plug-in whose host forbids device allocations outside the host's
// own API.  For them this entry point runs the same per-slice kernels as
// fv_execute but takes every piece of per-slice scratch memory (spreading
// grid, FFT band buffers, source bins and prepared sources, unique-target
// values) from one file-scope __device__ array of FV_STATIC_SCRATCH_BYTES
// that is part of the library image.  The call itself allocates nothing: no
// cudaMalloc, cudaFree, cudaMallocAsync or allocating library routine.
//
// The array is reserved on every device that loads this library's kernels,
// for the life of the process.  Its device address is looked up once per
// device (cudaGetSymbolAddress) by the first fv_execute_static call made on
// that device.
#include "fv_plan.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>

using namespace fv;

// Scratch shared by every fv_execute_static call on a device.
static __device__ __align__(256) unsigned char fv_static_scratch[FV_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
void *g_scratch_addr[64] = {};

// Device address of fv_static_scratch on `dev` (which must be current).
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void *a = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, fv_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = a;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carve {
    char *base;
    size_t used = 0;
    template <class T> T *take(size_t count)
    {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

struct Scratch {
    void *grid, *bufA, *bufB;
    cpx<double> *Vu;
    int *bin_of, *counts, *offsets, *cursor, *sidx, *cell;
    double *sdir;
    void *frac, *cs;
};

size_t layout(const fv_plan_s *p, char *base, Scratch &s)
{
    Carve c{base};
    const size_t es = p->elem(), gs = p->precision == FV_FP64 ? sizeof(double) : sizeof(float);
    s.grid = c.take<char>(std::max<size_t>(p->grid_elems, 1) * es);
    s.bufA = c.take<char>(std::max<size_t>(p->bufA_elems, 1) * es);
    s.bufB = c.take<char>(std::max<size_t>(p->bufB_elems, 1) * es);
    s.Vu = c.take<cpx<double>>(std::max<size_t>((size_t)p->n_u * p->n_pol, 1));
    if (p->tiled) {
        const size_t ns = std::max<long>(p->n_src, 1), nb = (size_t)p->nbx * p->nby;
        s.bin_of = c.take<int>(ns);
        s.counts = c.take<int>(nb);
        s.offsets = c.take<int>(nb + 1);
        s.cursor = c.take<int>(nb);
        s.sidx = c.take<int>(ns);
        s.cell = c.take<int>(3 * ns);
        s.sdir = c.take<double>(3 * ns);
        s.frac = c.take<char>(3 * ns * gs);
        s.cs = c.take<char>((size_t)p->n_pol * ns * es);
    }
    return c.used;
}

#define CKS(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string(#call " failed: ") + cudaGetErrorString(e_)); \
    } while (0)

template <class G>
fv_status run_static(fv_plan_s *p, const Scratch &sc, char *vis, size_t slice_bytes)
{
    const int nf = (int)p->freq.size(), nt = (int)p->lst.size();
    cpx<G> *grid = (cpx<G> *)sc.grid, *A = (cpx<G> *)sc.bufA, *Bb = (cpx<G> *)sc.bufB;
    const int nb = p->nbx * p->nby;
    const G *pre = (const G *)p->d_pre;
    const cpx<G> *tw = (const cpx<G> *)p->d_tw;
    for (int t = 0; t < nt; ++t) {
        TimeBin tb{};
        if (p->tiled) {
            std::memcpy(tb.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
            for (int i = 0; i < 3; ++i) {
                tb.C[i] = p->C[i];
                tb.qscale_top[i] = p->qscale_top[i];
                tb.nf1_top[i] = p->nf1_top[i];
            }
            tb.T[0] = p->T[0];
            tb.T[1] = p->T[1];
            tb.nbx = p->nbx;
            tb.nby = p->nby;
            // bin counts are cleared inside launch_time_binning on every call
            CKS(launch_time_binning(p->d_e, p->n_src, tb, sc.bin_of, sc.counts, sc.offsets, sc.cursor, sc.sdir,
                                    sc.sidx, p->stream));
        }
        for (int f = 0; f < nf; ++f) {
            SliceGeom g = p->gf[f];
            std::memcpy(g.R, &p->Rt[(size_t)t * 9], 9 * sizeof(double));
            const DimGeom *D = g.dim;
            const size_t o0 = (size_t)f * 3;
            if (p->tiled) {
                CKS(launch_prep<G>(sc.sdir, sc.sidx, sc.offsets + nb, p->n_src, p->flux, p->flux_fp64, nf, f, g,
                                   sc.cell, (G *)sc.frac, (cpx<G> *)sc.cs, p->stream));
                const double r0 = D[0].qscale / p->qscale_top[0], r1 = D[1].qscale / p->qscale_top[1];
                // every grid cell is stored by exactly one tile: no clearing needed
                if (p->spread_method == FV_SPREAD_SCATTER)
                    CKS(launch_spread_scatter<G>(sc.offsets, sc.cell, (const G *)sc.frac, (const cpx<G> *)sc.cs,
                                                 p->n_src, g, tb, r0, r1, grid, p->stream));
                else
                    CKS(launch_spread_tile<G>(sc.offsets, sc.cell, (const G *)sc.frac, (const cpx<G> *)sc.cs, p->n_src,
                                              g, tb, r0, r1, grid, p->stream));
            } else {
                // the atomic spreader accumulates: the grid must start at zero
                const size_t gel = (size_t)p->n_pol * D[0].nf1 * D[1].nf1 * D[2].nf1;
                CKS(cudaMemsetAsync(grid, 0, gel * sizeof(cpx<G>), p->stream));
                CKS(launch_spread_direct<G>(p->d_e, p->n_src, p->flux, p->flux_fp64, nf, f, g, grid, p->stream));
            }
            CKS(launch_fft_pass<G>(grid, A, (long)p->n_pol * D[2].nf1 * D[1].nf1, D[0], pre + p->pre_off[o0],
                                   tw + p->tw_off[o0], p->stream));
            CKS(launch_fft_pass<G>(A, Bb, (long)D[0].B * p->n_pol * D[2].nf1, D[1], pre + p->pre_off[o0 + 1],
                                   tw + p->tw_off[o0 + 1], p->stream));
            if (p->d == 2 || D[2].nf1 <= FV_ZDIRECT_MAX) {
                CKS(launch_interp_zdirect<G>(Bb, p->d_bu, p->n_u, p->d_dec, g, pre + p->pre_off[o0 + 2],
                                             tw + p->tw_off[o0 + 2], sc.Vu, p->stream));
            } else {
                CKS(launch_fft_pass<G>(Bb, A, (long)D[1].B * D[0].B * p->n_pol, D[2], pre + p->pre_off[o0 + 2],
                                       tw + p->tw_off[o0 + 2], p->stream));
                CKS(launch_interp<G>(A, p->d_bu, p->n_u, p->d_dec, g, sc.Vu, p->stream));
            }
            CKS(launch_scatter(sc.Vu, p->d_bl2u, p->n_bl, p->n_pol, vis + ((size_t)f * nt + t) * slice_bytes,
                               p->precision == FV_FP64, p->stream));
        }
    }
    return FV_OK;
}

}  // namespace

extern "C" fv_status fv_execute_static(fv_plan_t p, void *vis)
{
    if (!p) return FV_ERR_ARG;
    if (!vis) return p->fail(FV_ERR_ARG, "vis is NULL");
    if (!p->have_array || !p->have_sky) return p->fail(FV_ERR_STATE, "fv_set_array and fv_set_sky must come first");
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, vis) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return p->fail(FV_ERR_ARG, "fv_execute_static needs a device output buffer");
    }
    Scratch sc{};
    const size_t need = layout(p, nullptr, sc);
    if (need > FV_STATIC_SCRATCH_BYTES)
        return p->fail(FV_ERR_UNSUPPORTED, "this plan needs " + std::to_string(need) +
                                               " bytes of scratch; the static scratch holds " +
                                               std::to_string((size_t)FV_STATIC_SCRATCH_BYTES) + " bytes");
    void *base = nullptr;
    cudaError_t e = scratch_address(p->device, &base);
    if (e != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    layout(p, (char *)base, sc);
    const size_t cb = p->precision == FV_FP64 ? 16 : 8;
    const size_t slice_bytes = (size_t)p->n_bl * p->n_pol * cb;
    if (!p->any_visible || p->n_src == 0) {
        CKS(cudaMemsetAsync(vis, 0, slice_bytes * p->freq.size() * p->lst.size(), p->stream));
        return FV_OK;
    }
    return p->precision == FV_FP64 ? run_static<double>(p, sc, (char *)vis, slice_bytes)
                                   : run_static<float>(p, sc, (char *)vis, slice_bytes);
}
