// Prior simulation on the device (Table 1): theta_i = m_i + s_i z_i with z_i
// standard normal, a component with a finite lower bound (theta_8i >= -3)
// redrawn until it is inside (truncation by rejection).  Component i of
// particle n at attempt a takes normal i % 4 of the Philox4x64-10 block at
// counter (n, a, 0, 5 << 32 | i / 4) with key (seed, 0): Box-Muller on the
// 53-bit uniform pairs (0, 1) -> normals 0 (cosine), 1 (sine) and (2, 3) ->
// normals 2, 3.  After 64 rejected attempts the bound itself is used.
#include "../../include/smc.h"
#include "common.cuh"

namespace smc {

constexpr uint32_t kTagPrior = 5u;
constexpr int kPriorAttempts = 64;

struct PriorDev {
    int d;
    double mean[kMaxD], sd[kMaxD], lo[kMaxD];
};

__global__ void __launch_bounds__(256) k_draw_prior(PriorDev pr, uint64_t seed, int P, double* theta)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= P) return;
    const size_t Ps = (size_t)P;
    for (int i = 0; i < pr.d; ++i) {
        double x = pr.lo[i];
        for (int a = 0; a < kPriorAttempts; ++a) {
            const U64x4 r = philox4x64_10((uint64_t)n, (uint64_t)a, 0,
                                          ((uint64_t)kTagPrior << 32) | (uint64_t)(i / 4), seed, 0);
            const int pair = (i % 4) / 2;
            const uint64_t ua = pair == 0 ? r.v0 : r.v2, ub = pair == 0 ? r.v1 : r.v3;
            const double rho = sqrt(-2.0 * log(uniform53(ua)));
            double s, c;
            sincospi(2.0 * uniform53(ub), &s, &c);
            const double z = (i % 2 == 0) ? rho * c : rho * s;
            const double v = pr.mean[i] + pr.sd[i] * z;
            if (v >= pr.lo[i]) {
                x = v;
                break;
            }
        }
        theta[i * Ps + n] = x;
    }
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_draw_prior(const smc_model* m, uint64_t seed, int P, double* theta, void* stream)
{
    if (!m || !theta || P < 1) return SMC_EINVAL;
    const int d = m->n_free > 0 ? m->n_free : m->d_full;
    if (d < 1 || d > kMaxD) return SMC_EINVAL;
    PriorDev pr;
    pr.d = d;
    for (int i = 0; i < d; ++i) {
        if (!(m->prior_sd[i] > 0.0)) return SMC_EINVAL;
        pr.mean[i] = m->prior_mean[i];
        pr.sd[i] = m->prior_sd[i];
        pr.lo[i] = m->prior_lo[i];
    }
    k_draw_prior<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(pr, seed, P, theta);
    return cudaGetLastError() == cudaSuccess ? SMC_OK : SMC_ECUDA;
}
