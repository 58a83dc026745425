// Check of the bounded waits (no counterpart in the paper).  The spreading kernels wait on mbarrier phases
// for their bulk copies; every such wait gives up after about a second, records FV_DEVICE_TIMEOUT in the
// plan's status word and lets the kernel return, and the plan's next execution reports FV_ERR_TIMEOUT.
// fv_selftest_wait runs that path on purpose without any fault: one warp waits on a barrier phase that
// nothing completes (no copy is issued, nothing arrives), its wait runs out, and the result goes into the
// plan's status word exactly as a spreading kernel's would.
#include "fv_plan.cuh"
#include "fv_staged.cuh"

#include <string>

using namespace fv;

namespace {

__global__ void k_wait_selftest(int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init1(&bar);
    __syncwarp();
    // phase 0 of the barrier never completes: the bounded wait gives up
    const bool got = __all_sync(0xffffffffu, mbar_wait(&bar, 0u));
    if (!got && threadIdx.x == 0) atomicOr(status, FV_DEVICE_TIMEOUT);
}

}  // namespace

extern "C" fv_status fv_selftest_wait(fv_plan_t p)
{
    if (!p) return FV_ERR_ARG;
    if (cudaSetDevice(p->device) != cudaSuccess) return p->fail(FV_ERR_CUDA, "cudaSetDevice failed");
    k_wait_selftest<<<1, 32, 0, p->stream>>>(p->d_status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = plan_post_status(p);
    if (e != cudaSuccess) return p->fail(FV_ERR_CUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
    return FV_OK;
}
