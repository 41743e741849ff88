// Peak-rate microbenchmark of the pipes the likelihood recursion runs on.
//
// The M-phase kernels are bound by plain ALU work (the FP32 pipe, the SFU's
// ex2/lg2 and the instruction issue slot), not by HBM or tensor cores, so
// their roofline needs the rates of those pipes on the part at hand.  Each
// test is one launch of one 1024-thread block per SM (32 warps; each block
// asks for more than half of the SM's shared memory, so no SM can hold two
// and every SM gets exactly one); every thread runs kChains independent dependency
// chains of one operation, so that latency is hidden and the pipe's
// throughput is what is timed.  Every block records its SM's cycle counter
// and the global nanosecond timer around its loop: the SM clock during the
// test is cycles / ns, and the rate per SM and clock is the lane operations
// done / (SMs x cycles of the longest block).
//   FFMA   fma.rn.f32 (one lane operation per thread instruction)
//   FFMA2  fma.rn.f32x2 (Blackwell's paired FP32 instruction: two lane
//          operations per thread instruction)
//   EX2    ex2.approx.ftz.f32        LG2  lg2.approx.ftz.f32
//   DFMA   fma.rn.f64
//   ISSUE  an FFMA and a logic operation on its result in turn (two
//          instructions on different pipes): warp instructions issued per SM
//          and clock
//   MIX    an FFMA2 and an FFMA on independent chains in turn: FP32 lane
//          operations per SM and clock when paired and single instructions
//          share the FP32 pipes
// The loop body holds kReps x kChains operations, so that the loop's own
// counter and branch take about 1% of the issue slots.
#include "../../include/smc.h"
#include "common.cuh"

#include <vector>

namespace smc {

constexpr int kPeakThreads = 1024;
constexpr int kPeakSmem = 150 * 1024;   // > half of an SM's shared memory
constexpr int kChains = 8;
constexpr int kReps = 32;

enum { kOpFfma = 0, kOpFfma2, kOpEx2, kOpLg2, kOpDfma, kOpIssue, kOpMix, kNumOps };

struct PeakClock {
    unsigned long long cycles, ns;
};

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float a, float b, int* sink, PeakClock* clk)
{
    float x[kChains];
    double dx[kChains];
    unsigned int u[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = (float)(threadIdx.x + c) * 1e-3f;
        dx[c] = (double)x[c];
        u[c] = threadIdx.x * 7u + c;
    }
    float2 x2[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x2[c] = make_float2(x[c], x[c] + 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    const double da = (double)a, db = (double)b;
    __syncthreads();
    const unsigned long long c0 = clock64();
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int rep = 0; rep < kReps; ++rep) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP == kOpFfma) x[c] = fmaf(x[c], a, b);
                if constexpr (OP == kOpFfma2) x2[c] = __ffma2_rn(x2[c], a2, b2);
                if constexpr (OP == kOpEx2) x[c] = ex2_approx(-fabsf(x[c]));
                if constexpr (OP == kOpLg2) x[c] = lg2_approx(fabsf(x[c]) + b);
                if constexpr (OP == kOpDfma) dx[c] = fma(dx[c], da, db);
                if constexpr (OP == kOpIssue) {
                    x[c] = fmaf(x[c], a, b);
                    u[c] ^= __float_as_uint(x[c]);
                }
                if constexpr (OP == kOpMix) {
                    x2[c] = __ffma2_rn(x2[c], a2, b2);
                    x[c] = fmaf(x[c], a, b);
                }
            }
        }
    }
    const unsigned long long c1 = clock64();
    const unsigned long long t1 = global_ns();
    __syncthreads();
    float s = 0.0f;
    double ds = 0.0;
    unsigned int us = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        s += x[c] + x2[c].x + x2[c].y;
        ds += dx[c];
        us ^= u[c];
    }
    // keeps every chain live; the condition is never true for these inputs
    if (s == 1234.5f || ds == 1234.5 || us == 0x9e3779b9u) sink[0] = 1;
    if (threadIdx.x == 0) {
        clk[blockIdx.x].cycles = c1 - c0;
        clk[blockIdx.x].ns = t1 - t0;
    }
}

template <int OP>
static cudaError_t run_peak(int blocks, int iters, int* sink, PeakClock* clk, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_peak<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem);
    if (e != cudaSuccess) return e;
    k_peak<OP><<<blocks, kPeakThreads, kPeakSmem, s>>>(iters, 0.999f, 1e-3f, sink, clk);
    return cudaGetLastError();
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_peaks(smc_peak_rates* out, void* stream)
{
    if (!out) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SMC_ECUDA;
    const int blocks = sms;
    int* sink = nullptr;
    PeakClock* clk = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(int)) != cudaSuccess) return SMC_ECUDA;
    if (cudaMalloc((void**)&clk, (size_t)blocks * sizeof(PeakClock)) != cudaSuccess) {
        cudaFree(sink);
        return SMC_ECUDA;
    }
    std::vector<PeakClock> h(blocks);
    // lane operations per thread per loop iteration, and iteration counts that
    // keep each launch near a millisecond at the nominal rates
    const int per_iter = kReps * kChains;
    const int iters[kNumOps] = {1024, 512, 128, 64, 16, 512, 384};
    const double lanes_per_instr[kNumOps] = {1, 2, 1, 1, 1, 1, 3};   // MIX: per FFMA2 + FFMA pair
    const double instr_per_op[kNumOps] = {1, 1, 1, 1, 1, 2, 2};
    double rate[kNumOps], mhz[kNumOps];
    smc_status st = SMC_OK;
    for (int op = 0; op < kNumOps && st == SMC_OK; ++op) {
        for (int rep = 0; rep < 2 && st == SMC_OK; ++rep) {   // the first launch warms up
            cudaError_t e;
            switch (op) {
            case kOpFfma: e = run_peak<kOpFfma>(blocks, iters[op], sink, clk, s); break;
            case kOpFfma2: e = run_peak<kOpFfma2>(blocks, iters[op], sink, clk, s); break;
            case kOpEx2: e = run_peak<kOpEx2>(blocks, iters[op], sink, clk, s); break;
            case kOpLg2: e = run_peak<kOpLg2>(blocks, iters[op], sink, clk, s); break;
            case kOpDfma: e = run_peak<kOpDfma>(blocks, iters[op], sink, clk, s); break;
            case kOpIssue: e = run_peak<kOpIssue>(blocks, iters[op], sink, clk, s); break;
            default: e = run_peak<kOpMix>(blocks, iters[op], sink, clk, s); break;
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), clk, (size_t)blocks * sizeof(PeakClock),
                                                      cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = SMC_ECUDA;
        }
        if (st != SMC_OK) break;
        unsigned long long cmax = 0;
        double ratio = 0.0;
        for (int b = 0; b < blocks; ++b) {
            cmax = h[b].cycles > cmax ? h[b].cycles : cmax;
            ratio += h[b].ns ? (double)h[b].cycles / (double)h[b].ns : 0.0;
        }
        // lane operations per SM per clock: every SM holds one block of
        // kPeakThreads threads, each doing iters x per_iter operations
        const double ops_per_sm = (double)kPeakThreads * (double)iters[op] * per_iter * lanes_per_instr[op];
        rate[op] = cmax ? ops_per_sm / (double)cmax : 0.0;
        // ISSUE: warp instructions per SM and clock
        if (op == kOpIssue) rate[op] = rate[op] * instr_per_op[op] / 32.0;
        mhz[op] = 1e3 * ratio / blocks;
    }
    cudaFree(sink);
    cudaFree(clk);
    if (st != SMC_OK) return st;
    out->sms = sms;
    out->ffma = rate[kOpFfma];
    out->ffma2 = rate[kOpFfma2];
    out->ex2 = rate[kOpEx2];
    out->lg2 = rate[kOpLg2];
    out->dfma = rate[kOpDfma];
    out->issue = rate[kOpIssue];
    out->ffma_mix = rate[kOpMix];
    double m = 0.0;
    for (int op = 0; op < kNumOps; ++op) m += mhz[op];
    out->sm_mhz = m / kNumOps;
    return SMC_OK;
}
