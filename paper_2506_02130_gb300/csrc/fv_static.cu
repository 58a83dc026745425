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
// The array is committed on a device when the module holding it is loaded
// there: with CUDA's lazy module loading (the default) that is the first
// fv_execute_static call on that device, which also looks up its device
// address (cudaGetSymbolAddress) once per device.  Callers holding a fixed
// HBM budget make one warm-up call (a tiny plan will do) before fixing it.
// The cached address belongs to the device's primary context: after a
// cudaDeviceReset in the same process the first call looks it up again.
#include "fv_plan.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

using namespace fv;

// Scratch shared by every fv_execute_static call on a device.
static __device__ __align__(256) unsigned char fv_static_scratch[FV_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
void *g_scratch_addr[64] = {};
unsigned long long g_scratch_ctx[64] = {};   // the primary context the address was looked up in

// Identifier of the current context (0 if the driver cannot say), through the driver's entry point.
unsigned long long current_context_id()
{
    using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);
    static CtxGetId fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetId)f;
        cudaGetLastError();
        looked = true;
    }
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of fv_static_scratch on `dev` (which must be current).
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    // a context created since (cudaDeviceReset) holds the array at another address: look it up again
    const unsigned long long ctx = current_context_id();
    if (g_scratch_addr[dev] && g_scratch_ctx[dev] != ctx) g_scratch_addr[dev] = nullptr;
    if (!g_scratch_addr[dev]) {
        void *a = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, fv_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = a;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

#define CKS(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string(#call " failed: ") + cudaGetErrorString(e_)); \
    } while (0)


extern "C" fv_status fv_execute_static(fv_plan_t p, void *vis)
{
    if (!p) return FV_ERR_ARG;
    if (!vis) return p->fail(FV_ERR_ARG, "vis is NULL");
    if (!p->have_array || !p->have_sky) return p->fail(FV_ERR_STATE, "fv_set_array and fv_set_sky must come first");
    if (p->use_basis) return p->fail(FV_ERR_UNSUPPORTED, "a spectral-basis plan runs through fv_execute only");
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, vis) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return p->fail(FV_ERR_ARG, "fv_execute_static needs a device output buffer");
    }
    if (pa.type == cudaMemoryTypeDevice && pa.device != p->device)
        return p->fail(FV_ERR_ARG, "the output buffer is on another device than the plan");
    if ((uintptr_t)vis % (p->precision == FV_FP64 ? 16u : 8u) != 0)
        return p->fail(FV_ERR_ARG, "vis must be aligned to its element size");
    fv_status prev = plan_take_status(p, false);
    if (prev != FV_OK) return prev;
    // the same carving as a plan's own execution workspace (fv_plan_s::need), over the static array
    const size_t need = workspace_layout(p->need, nullptr, nullptr);
    if (need > FV_STATIC_SCRATCH_BYTES)
        return p->fail(FV_ERR_UNSUPPORTED, "this plan needs " + std::to_string(need) +
                                               " bytes of scratch; the static scratch holds " +
                                               std::to_string((size_t)FV_STATIC_SCRATCH_BYTES) + " bytes");
    void *base = nullptr;
    cudaError_t e = scratch_address(p->device, &base);
    if (e != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    fv_plan_s::Workspace wk{};
    workspace_layout(p->need, (char *)base, &wk);
    const size_t cb = p->precision == FV_FP64 ? 16 : 8;
    const size_t slice_bytes = (size_t)p->n_bl * p->n_pol * cb;
    const long total = (long)p->freq.size() * p->lst.size();
    if (!p->any_visible || p->n_src == 0) {
        CKS(cudaMemsetAsync(vis, 0, slice_bytes * total, p->stream));
        return FV_OK;
    }
    // the channel-major flux copy (a plan-owned buffer made at fv_set_sky), then every slice on the plan's
    // stream, in order, through the one scratch workspace
    CKS(refresh_flux_t(p, p->stream));
    fv_status s = p->precision == FV_FP64 ? run_slices<double>(p, wk, p->stream, (char *)vis, slice_bytes, 0, total)
                                          : run_slices<float>(p, wk, p->stream, (char *)vis, slice_bytes, 0, total);
    if (s == FV_OK) CKS(plan_post_status(p));   // a copy of the status word into pinned memory: no allocation
    return s;
}
