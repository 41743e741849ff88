// Self-test of the bounded device waits (failure detection without a fault).
//
// Every wait of the library's kernels on an mbarrier is bounded in wall time;
// when the bound runs out the kernel records an error, lets its own copies
// land (again bounded) and returns, so the host sees SMC_ETIMEOUT and the
// context stays usable.  This entry point runs the same wait on a barrier that
// is completed only when `complete` is set, so a test can make the wait run
// out on purpose and check that the status comes back and later work runs.
#include "../../include/smc.h"
#include "common.cuh"

namespace smc {

__global__ void k_wait_selftest(uint64_t limit_ns, int complete, int* timed_out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && complete)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    const bool any_failed = __syncthreads_or(!ok);
    if (threadIdx.x == 0) {
        *timed_out = any_failed ? 1 : 0;
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar)) : "memory");
    }
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_wait_selftest(uint64_t limit_ns, int complete, void* stream)
{
    if (limit_ns == 0 || limit_ns > kWaitLimitNs) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int* flag = nullptr;
    if (cudaMallocAsync((void**)&flag, sizeof(int), s) != cudaSuccess) return SMC_ECUDA;
    k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, complete ? 1 : 0, flag);
    int h = -1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(flag, s);
    if (e != cudaSuccess) return SMC_ECUDA;
    return h == 1 ? SMC_ETIMEOUT : (h == 0 ? SMC_OK : SMC_ECUDA);
}
