// Covariance tile sums shared by the mutation kernel's epilogue and the S
// phase's gather.
#pragma once

#include <cstddef>

namespace smc {

// Row of entry q of the packed lower triangle (q = i(i+1)/2 + k, k <= i).
__host__ __device__ constexpr int tri_row(int q)
{
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    return i;
}

// Covariance tile sums of one warp's 32 consecutive particles (p is this
// lane's particle; lanes past P contribute zeros): S1_i (entry i) and S2_ik
// (entry kD + i(i+1)/2 + k, k <= i) of x_i = theta_i - shift_i in FP32, for
// the compile-time bound kD >= d (entries past d are zero).  The warp forms
// the products 16 entries at a time and reduce-scatters them in four halving
// levels and one exchange, after which lanes 2e and 2e + 1 hold entry e of the
// group: one shuffle per entry instead of five, with independent shuffles at
// each level.
// The tile is the same 32 particles in every launch shape, so the covariance
// does not depend on the shape.  theta is [d][P] (the particles after the
// decision, or after the S phase's gather); covtile is
// [kD + kD(kD+1)/2][ntiles].  Every lane of the warp calls it.
template <int kD>
__device__ __forceinline__ void cov_tile_sums(const double* __restrict__ theta, size_t P, int d,
                                              const float* __restrict__ covshift, float* __restrict__ covtile,
                                              int ntiles, int p, bool active)
{
    constexpr int kAcc = kD + kD * (kD + 1) / 2;
    constexpr int kGroups = (kAcc + 15) / 16;
    const int tile = p >> 5;
    if (tile >= ntiles) return;   // a whole warp past P (warp-uniform)
    const int lane = threadIdx.x & 31;
    float x[kD];
#pragma unroll
    for (int i = 0; i < kD; ++i) x[i] = (active && i < d) ? (float)theta[i * P + p] - covshift[i] : 0.0f;
    const size_t nt = (size_t)ntiles;
#pragma unroll
    for (int c = 0; c < kGroups; ++c) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int g = 16 * c + j;
            if (g < kD) {
                v[j] = x[g < kD ? g : 0];
            } else if (g < kAcc) {
                const int q = g - kD;
                const int i = tri_row(q), k = q - tri_row(q) * (tri_row(q) + 1) / 2;
                v[j] = x[i < kD ? i : 0] * x[k < kD ? k : 0];
            } else {
                v[j] = 0.0f;
            }
        }
        // four halving levels leave lane l with entry (l >> 1) summed over
        // 16 lanes; the last exchange adds the other half of the warp
#pragma unroll
        for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < n / 2; ++j) {
                const float keep = up ? v[j + n / 2] : v[j];
                const float send = up ? v[j] : v[j + n / 2];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
        const int g = 16 * c + (lane >> 1);
        if ((lane & 1) == 0 && g < kAcc) covtile[(size_t)g * nt + tile] = v[0];
    }
}

}  // namespace smc
