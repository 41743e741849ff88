// Device-side building blocks shared by the simulator kernels.
//
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from the
// published round function and key schedule; the counter map
//   key = (seed, 0), counter = (particle or group, iteration or draw, cycle,
//                               tag << 32 | block)
// gives every random number of a run a fixed address, so a run does not depend
// on the launch shape.  Uniforms are ((x >> 11) + 0.5) 2^-53.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smc {

constexpr int kMaxD = 32;       // free parameters carried by a particle
constexpr int kMaxK = 4;        // volatility factors
constexpr int kMaxI = 4;        // mixture components
constexpr int kMaxState = kMaxK + 1;
constexpr int kMaxN = 8192;      // particles per group (S-phase shared memory)

enum : uint32_t { kTagNormal = 1u, kTagUniform = 2u, kTagResample = 3u, kTagPit = 4u };

// ------------------------------------------------------------------ Philox4x64
struct U64x4 {
    uint64_t v0, v1, v2, v3;
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;   // round multipliers
    constexpr uint64_t kM1 = 0xCA5A826395121157ull;
    constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;   // Weyl key increments
    constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
        const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += kW0;
        k1 += kW1;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ double uniform53(uint64_t x)
{
    return ((double)(x >> 11) + 0.5) * 0x1.0p-53;
}

// Proposal normals for particle p at (cycle, iter): Box-Muller on the pairs
// (u0,u1), (u2,u3) of each Philox block b; normal 4b+2k uses cos, 4b+2k+1 sin.
template <typename Real>
__device__ __forceinline__ void proposal_normals(uint64_t seed, uint64_t p, uint64_t iter,
                                                 uint64_t cycle, int d, Real* z)
{
    for (int b = 0; 4 * b < d; ++b) {
        const U64x4 r = philox4x64_10(p, iter, cycle, ((uint64_t)kTagNormal << 32) | (uint64_t)b,
                                      seed, 0);
        const uint64_t u[4] = {r.v0, r.v1, r.v2, r.v3};
#pragma unroll
        for (int pair = 0; pair < 2; ++pair) {
            const int n = 4 * b + 2 * pair;
            if (n >= d) break;
            if constexpr (sizeof(Real) == 8) {
                const double ua = uniform53(u[2 * pair]), ub = uniform53(u[2 * pair + 1]);
                const double rho = sqrt(-2.0 * log(ua));
                double s, c;
                sincospi(2.0 * ub, &s, &c);
                z[n] = rho * c;
                if (n + 1 < d) z[n + 1] = rho * s;
            } else {
                // 24-bit uniforms ((x >> 40) + 1/2) 2^-24: the same draws as the
                // 53-bit ones to FP32 precision, without FP64 conversions
                const float ua = ((float)(uint32_t)(u[2 * pair] >> 40) + 0.5f) * 0x1.0p-24f;
                const float ub = ((float)(uint32_t)(u[2 * pair + 1] >> 40) + 0.5f) * 0x1.0p-24f;
                const float rho = sqrtf(-2.0f * logf(ua));
                float s, c;
                sincospif(2.0f * ub, &s, &c);
                z[n] = rho * c;
                if (n + 1 < d) z[n + 1] = rho * s;
            }
        }
    }
}

__device__ __forceinline__ double log_uniform_mh(uint64_t seed, uint64_t p, uint64_t iter,
                                                 uint64_t cycle)
{
    const U64x4 r = philox4x64_10(p, iter, cycle, (uint64_t)kTagUniform << 32, seed, 0);
    return log(uniform53(r.v0));
}

// Metropolis-Hastings decision log u < log_alpha for the uniform of
// log_uniform_mh, without the FP64 logarithm in nearly all cases: the log of
// the 24-bit uniform u24 (the centre of the 2^-24 interval holding the 53-bit
// uniform, so |u24 - u53| <= 2^-25) is within 3e-5 of log u53 when
// u24 >= 2^-10, and the FP32 logarithm and rounding of log_alpha add at most
// ~1e-6 while |log_alpha| < 20 (beyond that the margin is large).  A decision
// more than 1e-3 from the threshold is therefore the FP64 decision; the rest,
// and u24 < 2^-10, take the FP64 logarithm.  A NaN log_alpha rejects.
__device__ __forceinline__ bool mh_accept(uint64_t seed, uint64_t p, uint64_t iter, uint64_t cycle,
                                          double log_alpha)
{
    const U64x4 r = philox4x64_10(p, iter, cycle, (uint64_t)kTagUniform << 32, seed, 0);
    const float u24 = ((float)(uint32_t)(r.v0 >> 40) + 0.5f) * 0x1.0p-24f;
    const float lu = __logf(u24);
    const float la = (float)log_alpha;
    if (u24 >= 0x1.0p-10f && fabsf(lu - la) > 1e-3f) return lu < la;
    return log(uniform53(r.v0)) < log_alpha;
}

// ------------------------------------------------------------ SFU instructions
// Hardware base-2 exponential / logarithm (PTX ex2.approx / lg2.approx, flush
// to zero).  Used only on the FP32 path, whose tolerance against the FP64
// oracle is 1e-4 relative.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ----------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum with a fixed combination order (deterministic).  scratch
// holds at least 32 elements; all threads receive the result.
template <typename T>
__device__ T block_sum(T v, T* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T r = (threadIdx.x < (unsigned)nwarps) ? scratch[threadIdx.x] : T(0);
    if (warp == 0) r = warp_sum(r);
    if (threadIdx.x == 0) scratch[0] = r;
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

// Inclusive block scan of one value per thread (u64).  scratch >= 32 elements.
__device__ inline uint64_t block_inclusive_scan_u64(uint64_t v, uint64_t* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    __syncthreads();
    if (lane == 31) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = (lane < nwarps) ? scratch[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nwarps) scratch[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += scratch[warp - 1];
    __syncthreads();
    return v;
}

// ------------------------------------------------- mbarrier + bulk async copy
// Observation staging uses the Blackwell bulk-copy engine (cp.async.bulk, the
// non-tensor form of TMA) completing on an mbarrier.  Every wait is bounded in
// wall time (kWaitLimitNs on the global nanosecond timer): when it runs out the
// wait reports failure and the caller records an error instead of hanging.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Programmatic dependent launch (PTX griddepcontrol): a kernel launched with
// pdl_launch may start while its predecessor in the stream is still running.
// pdl_wait() returns once the predecessor has completed and its writes are
// visible (at once when there is no such predecessor), so a kernel calls it
// before touching anything a preceding kernel writes; pdl_trigger() lets the
// next kernel launch once every block of this one has passed it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Error word bits reported through the context.
enum : int { kErrTimeout = 1, kErrNonFinite = 2, kErrDegenerate = 4, kErrBounds = 8 };

__device__ __forceinline__ void raise_error(int* err, int bits)
{
    if (err) atomicOr(err, bits);
}

}  // namespace smc
