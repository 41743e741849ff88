// smc_cov_chol_noalloc: the pooled covariance + Cholesky entry point without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: a host framework
// that reserves the whole device memory budget up front and hands out only
// pre-sized buffers, or a latency-bound loop in which a stream-ordered
// allocation could wait on the memory pool.  For them this variant takes its
// partial-sum scratch from a fixed array compiled into the library instead of
// cudaMallocAsync.  The caller still passes theta and the outputs.
//
// The scratch is one file-scope __device__ array, so every process that loads
// the library holds it on every device it uses until exit (about 2.3 MB).
// All calls on a device share it and it keeps the last call's contents: each
// call writes every partial sum it later reads, and the reduction's counter in
// the last element returns to zero at the end of each call, so nothing needs
// clearing; but two calls whose kernels overlap on the GPU (different streams
// without ordering between them) race on it and must not be issued.
// Back-to-back calls on one stream are ordered although the reduction kernel
// lets the next launch start early (programmatic dependent launch): both the
// partial-sum kernel and the reduction wait for their predecessor
// (griddepcontrol.wait) before their first access to the array, and any kernel
// added to this path must do the same.
// The block count is the allocating entry point's (cov_grid: at most two blocks
// per SM), so on any device with up to 256 SMs both split the particles the
// same way and their results are identical; beyond that it is capped at
// kNoAllocCovBlocks and the results agree within FP rounding of the sums.
#include "../../include/smc.h"
#include "phase.cuh"

#include <mutex>

namespace smc {

// Block partials of the covariance kernel: at most kNoAllocCovBlocks blocks
// plus one row of totals, each row holding d + d(d+1)/2 sums for d <= kMaxD.
constexpr int kNoAllocCovBlocks = 512;
constexpr int kNoAllocCovRow = kMaxD + kMaxD * (kMaxD + 1) / 2;
constexpr size_t kNoAllocScratchDoubles = (size_t)(kNoAllocCovBlocks + 1) * kNoAllocCovRow;

// The element after the partial sums holds the reduction's counter (zero
// while no call runs: device memory starts zeroed and each call resets it).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles + 1];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ variable is only a stand-in, so the address is looked up
// once per device (with that device current) and cached.  The cache assumes the
// device's context lives as long as the process: after cudaDeviceReset (which
// unloads the module holding the array) the cached address is stale, so this
// entry point must not be called again in that process.
cudaError_t scratch_on_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace smc

using namespace smc;

extern "C" smc_status smc_cov_chol_noalloc(const double* theta, int d, int P, int h_tenths,
                                           double* mean, double* cov, double* L, void* stream)
{
    if (!theta || d < 1 || d > SMC_MAX_D || P < 2 || h_tenths < 0) return SMC_EINVAL;
    double* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return SMC_ECUDA;
    int G = cov_grid(P);
    if (G > kNoAllocCovBlocks) G = kNoAllocCovBlocks;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocScratchDoubles);
    const cudaError_t e = launch_cov(theta, d, P, scratch, G, counter, nullptr, h_tenths, 0.0, 1, 10, mean,
                                     cov, L, (cudaStream_t)stream);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}
