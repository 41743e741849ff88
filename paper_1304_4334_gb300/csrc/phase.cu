// C-phase search, S phase, covariance/Cholesky and estimator kernels.
#include "phase.cuh"
#include "covtile.cuh"
#include "exp2_table.h"

#include <cstdio>

namespace smc {

extern void count_launch();

int device_sm_count()
{
    static int cached = 0;
    if (!cached) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached = n > 0 ? n : 1;
    }
    return cached;
}

// ============================================================ covariance
// V_lr of Section 3.3 is the sample variance of the current particles, pooled
// over all J N.  Sums are taken about a shift (particle 0) so that the final
// combination does not cancel: V = [S2 - S1 S1'/P] / (P - 1) on shifted data.
// Within a tile of 64 particles the shifted values and their products are
// summed in FP32 (the FP64 pipe of this part is 1/64 of its FP32 rate); tiles
// and blocks are combined in FP64.  V only scales the random-walk proposal, so
// its ~1e-6 relative accuracy leaves the Metropolis kernel exact.
constexpr int kCovThreads = 256;
constexpr int kCovTile = 64;
constexpr int kCovMaxAcc = (kMaxD + kMaxD * (kMaxD + 1) / 2 + kCovThreads - 1) / kCovThreads;

int cov_grid(int P)
{
    const int by_tiles = (P + kCovTile - 1) / kCovTile;
    const int cap = 2 * device_sm_count();
    return by_tiles < cap ? by_tiles : cap;
}

__device__ __forceinline__ void unpack_pair(int e, int& i, int& k)
{
    // e = i (i + 1) / 2 + k, 0 <= k <= i
    int ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
    while (ii * (ii + 1) / 2 > e) --ii;
    i = ii;
    k = e - ii * (ii + 1) / 2;
}

__device__ void cov_partial_body(const double* __restrict__ theta, int d, int P,
                                 double* __restrict__ part, int bidx, int G)
{
    __shared__ float tile[kMaxD][kCovTile + 1];
    __shared__ double shift[kMaxD];
    __shared__ int pi_[kMaxD * (kMaxD + 1) / 2], pk_[kMaxD * (kMaxD + 1) / 2];
    const int npair = d * (d + 1) / 2;
    const int nacc = d + npair;
    const size_t Ps = (size_t)P;
    for (int e = threadIdx.x; e < npair; e += blockDim.x) unpack_pair(e, pi_[e], pk_[e]);
    for (int i = threadIdx.x; i < d; i += blockDim.x) shift[i] = theta[i * Ps];
    double acc[kCovMaxAcc];
#pragma unroll
    for (int r = 0; r < kCovMaxAcc; ++r) acc[r] = 0.0;
    const int per = (P + G - 1) / G;
    const int n0 = bidx * per;
    const int n1 = min(P, n0 + per);
    __syncthreads();
    for (int base = n0; base < n1; base += kCovTile) {
        const int cnt = min(kCovTile, n1 - base);
        for (int e = threadIdx.x; e < d * kCovTile; e += blockDim.x) {
            const int i = e / kCovTile, n = e % kCovTile;
            tile[i][n] = n < cnt ? (float)(theta[i * Ps + base + n] - shift[i]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kCovMaxAcc; ++r) {
            const int e = threadIdx.x + r * blockDim.x;
            if (e < d) {
                float s = 0.0f;
                for (int n = 0; n < cnt; ++n) s += tile[e][n];
                acc[r] += (double)s;
            } else if (e < nacc) {
                const int i = pi_[e - d], k = pk_[e - d];
                float s = 0.0f;
                for (int n = 0; n < cnt; ++n) s = fmaf(tile[i][n], tile[k][n], s);
                acc[r] += (double)s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < kCovMaxAcc; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        if (e < nacc) part[(size_t)bidx * nacc + e] = acc[r];
    }
}

__global__ void __launch_bounds__(kCovThreads) k_cov_partial(const double* __restrict__ theta, int d,
                                                            int P, double* __restrict__ part)
{
    pdl_trigger();
    pdl_wait();
    cov_partial_body(theta, d, P, part, blockIdx.x, gridDim.x);
}

__device__ void apply_h_update(Ctl* ctl, int P, double target, int hmin, int hmax)
{
    if (ctl->pending) {
        const double rate = (double)ctl->acc_count / (double)P;
        int h = ctl->h_tenths + (rate > target ? 1 : -1);
        h = h < hmin ? hmin : (h > hmax ? hmax : h);
        ctl->h_tenths = h;
        ctl->acc_sum += rate;
        ctl->acc_n += 1;
        ctl->acc_count = 0ull;
        ctl->pending = 0;
    }
}

__global__ void k_adapt_h(Ctl* ctl, int P, double target, int hmin, int hmax)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) apply_h_update(ctl, P, target, hmin, hmax);
}



// ---- double-float arithmetic for the factorisation (value = hi + lo) ----
// Error-free transformations on the FP32 pipe (Knuth's TwoSum, Dekker's
// product through fmaf) carry about 44 significant bits at FP32 latency; on
// this part an FP64 instruction holds its pipe for ~64 cycles.  Products that
// feed an addition use __fmul_rn, which the compiler never fuses into an FMA
// (a fused rounding would break the exact error terms).
struct Df {
    float hi, lo;
};

__device__ __forceinline__ Df df_quick(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ Df df_mul(Df x, Df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return df_quick(p, e);
}

// a - x y
__device__ __forceinline__ Df df_fms(Df a, Df x, Df y)
{
    const Df p = df_mul(x, y);
    const float s = a.hi - p.hi;
    const float bv = s - a.hi;
    float e = (a.hi - (s - bv)) + (-p.hi - bv);
    e += a.lo - p.lo;
    return df_quick(s, e);
}

// p^-1/2 for p > 0: the FP32 reciprocal square root y0 (about 22 correct
// bits) refined by one Newton step y0 + (y0/2)(1 - p y0^2), the residual
// formed from exact products (about 43 bits, 1e-13 relative).
__device__ __forceinline__ Df df_rsqrt(Df p)
{
    const float y0 = rsqrtf(p.hi);
    const float q = __fmul_rn(y0, y0);
    const float qe = fmaf(y0, y0, -q);        // y0^2 = q + qe
    const float t = __fmul_rn(p.hi, q);
    const float te = fmaf(p.hi, q, -t);       // p.hi q = t + te
    const float r = ((1.0f - t) - te) - fmaf(p.hi, qe, __fmul_rn(p.lo, q));
    return df_quick(y0, __fmul_rn(__fmul_rn(0.5f, y0), r));
}

__device__ __forceinline__ double pow2(int m)   // 2^m, |m| <= 1022
{
    return __longlong_as_double((long long)(1023 + m) << 52);
}

// Final step of the covariance (one block): updates h from the previous
// iteration's acceptance (when a control block is given; a positive fixed_h
// still scales Sigma in place of the adapted h), forms V from the totals of
// the shifted sums and factors Sigma = h^2 V as h chol(V), a non-positive
// pivot zeroing its column, as in the oracle.  The factorisation runs on
// S = D V D, D = diag(2^-m_i) with 2^(2 m_i) near V_ii (exact scaling, unit-
// sized entries), in double-float arithmetic by the first warp with element
// indices from a table; chol(V) = D^-1 chol(S).  A pivot of S below 1e-30
// (relative to its unit-sized diagonal: far below the rounding of V's sums)
// counts as zero.
// The shift of the sums is shift_f[i] (FP32, the mutation tiles) when given,
// else shift_in[i * shift_stride]; the pooled mean goes to mean_out (FP64)
// and, rounded, to mean_f_out (the next tiles' shift; may be shift_f).  The
// divisions and the step-size update run on separate warps while the totals
// load.
constexpr int kMaxPair = kMaxD * (kMaxD + 1) / 2;

__device__ void cov_final_body(const double* __restrict__ tot, int d, int P,
                               const double* __restrict__ shift_in, size_t shift_stride,
                               const float* shift_f, Ctl* ctl, int fixed_h, double target, int hmin,
                               int hmax, double* mean_out, float* mean_f_out, double* cov_out,
                               double* L_out)
{
    __shared__ double S1[kMaxD];
    __shared__ double A[kMaxD][kMaxD + 1];
    __shared__ Df F[kMaxD][kMaxD + 1];
    __shared__ double shift[kMaxD];
    __shared__ int msc[kMaxD];
    __shared__ unsigned char pi_[kMaxPair], pk_[kMaxPair];
    __shared__ double hs, invP, invP1;
    const int npair = d * (d + 1) / 2;
    if (threadIdx.x == 0) {
        invP = 1.0 / (double)P;
    } else if (threadIdx.x == 32) {
        invP1 = 1.0 / (double)(P - 1);
    } else if (threadIdx.x == 64) {
        int h = fixed_h;
        if (ctl) {
            apply_h_update(ctl, P, target, hmin, hmax);
            if (fixed_h <= 0) h = ctl->h_tenths;   // fixed_h > 0 overrides the adapted step size
        }
        hs = h / 10.0;
    }
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        int i, k;
        unpack_pair(e, i, k);
        pi_[e] = (unsigned char)i;
        pk_[e] = (unsigned char)k;
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x)
        shift[i] = shift_f ? (double)shift_f[i] : shift_in[i * shift_stride];
    for (int e = threadIdx.x; e < d; e += blockDim.x) S1[e] = __ldcg(tot + e);
    __syncthreads();
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        const int i = pi_[e], k = pk_[e];
        const double c = (__ldcg(tot + d + e) - S1[i] * S1[k] * invP) * invP1;
        A[i][k] = c;
        A[k][i] = c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) {   // the shifts are in shared memory already
        const double mu = shift[i] + S1[i] * invP;
        if (mean_out) mean_out[i] = mu;
        if (mean_f_out) mean_f_out[i] = (float)mu;
        // m_i = floor(e_i / 2) for V_ii = 2^e_i * 1.f (positive normal), else 0
        const long long b = __double_as_longlong(A[i][i]);
        msc[i] = (b > 0x000fffffffffffffLL && b < 0x7ff0000000000000LL) ? (((int)(b >> 52) - 1023) >> 1) : 0;
    }
    if (cov_out)
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) cov_out[e] = A[e / d][e % d];
    __syncthreads();
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        const int i = pi_[e], k = pk_[e];
        const double sik = A[i][k] * pow2(-(msc[i] + msc[k]));
        const float hi = __double2float_rn(sik);
        F[i][k] = {hi, __double2float_rn(sik - (double)hi)};
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = 0; j < d; ++j) {
            const Df piv = F[j][j];
            Df y = {0.0f, 0.0f};
            if (piv.hi > 1e-30f) y = df_rsqrt(piv);
            // lane j forms sqrt(piv) = piv y, lanes below it l_ij = s_ij y
            const bool col = lane >= j && lane < d;
            Df v = {0.0f, 0.0f};
            if (col) v = df_mul(F[lane][j], y);
            __syncwarp();
            if (col) F[lane][j] = v;
            __syncwarp();
            const int m = d - j - 1;
            const int ne = m * (m + 1) / 2;
            for (int e = lane; e < ne; e += 32) {
                const int ii = pi_[e] + j + 1, kk = pk_[e] + j + 1;
                F[ii][kk] = df_fms(F[ii][kk], F[ii][j], F[kk][j]);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (L_out)
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
            const int i = e / d, k = e % d;
            L_out[e] = k <= i ? ((double)F[i][k].hi + (double)F[i][k].lo) * (hs * pow2(msc[i])) : 0.0;
        }
}

// Totals of the partial sums (one block per entry, fixed order), then the
// final step in the last block to finish (the counter returns to zero for the
// next launch).  Partials: kTiles, FP32 tile sums [nacc][nparts]; otherwise
// FP64 block sums [nparts][nacc].
struct CovFinalArgs {
    int d, P;
    const double* shift_in;
    long long shift_stride;
    const float* shift_f;
    Ctl* ctl;
    int fixed_h;
    double target;
    int hmin, hmax;
    double* mean_out;
    float* mean_f_out;
    double *cov_out, *L_out;
    int tile_kd;   // tile layout bound (tiles only)
};

// Total of entry e over the partials, kCovThreads threads in a fixed order
// (the single-run and batched paths share it, so their sums agree bitwise).
// For tiles, entry e of the d-layout is row e (e < d) or e - d + kD of the
// tiles' kD-layout.
template <bool kTiles>
__device__ __forceinline__ double cov_entry_total(const void* __restrict__ parts, int nparts, int nacc, int e,
                                                  int d, int kD, double* red)
{
    double s = 0.0;
    if constexpr (kTiles) {
        // Runs of 16 tile sums are added in FP32 with the rounding error of
        // every addition carried along (Knuth's TwoSum), so each run enters
        // FP64 as an almost exact pair: a sixteenth of the FP64 additions
        // (each FP64 instruction holds its pipe for about 64 cycles here), with
        // no loss against summing every tile in FP64.  A thread issues all
        // loads of a run before it adds (16-byte loads when rows allow).
        const int r = e < d ? e : e - d + kD;
        const float* row = static_cast<const float*>(parts) + (size_t)r * nparts;
        float hi = 0.0f, lo = 0.0f;
        auto add = [&](float v) {
            const float a = hi + v;
            const float bv = a - hi;
            lo += (hi - (a - bv)) + (v - bv);
            hi = a;
        };
        auto flush = [&]() {
            s += (double)hi + (double)lo;
            hi = lo = 0.0f;
        };
        const int nb = blockDim.x;
        if ((nparts & 3) == 0) {
            const float4* row4 = reinterpret_cast<const float4*>(row);
            const int n4 = nparts >> 2;
            for (int t0 = threadIdx.x; t0 < n4; t0 += 4 * nb) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    v[u] = t0 + u * nb < n4 ? row4[t0 + u * nb] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    add(v[u].x);
                    add(v[u].y);
                    add(v[u].z);
                    add(v[u].w);
                }
                flush();
            }
        } else {
            for (int t0 = threadIdx.x; t0 < nparts; t0 += 16 * nb) {
                float v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = t0 + u * nb < nparts ? row[t0 + u * nb] : 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u) add(v[u]);
                flush();
            }
        }
    } else {
        const double* pp = static_cast<const double*>(parts);
        for (int g = threadIdx.x; g < nparts; g += blockDim.x) s += pp[(size_t)g * nacc + e];
    }
    return block_sum(s, red);
}

template <bool kTiles>
__global__ void __launch_bounds__(kCovThreads) k_cov_reduce(const void* __restrict__ parts, int nparts,
                                                            int nacc, double* tot, unsigned int* counter,
                                                            CovFinalArgs f)
{
    __shared__ double red[32];
    __shared__ int last;
    pdl_wait();
    const int e = blockIdx.x;
    const double s = cov_entry_total<kTiles>(parts, nparts, nacc, e, f.d, f.tile_kd, red);
    if (threadIdx.x == 0) {
        tot[e] = s;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // Every other block has left: the mutation kernel that follows (a
    // dependent launch) may now place its blocks, evenly over the nearly empty
    // SMs, and they wait for this block's factor.  (Placed earlier, while the
    // SMs were still unevenly busy, they landed unevenly and the one-wave
    // kernel ran as long as its most loaded SM.)
    pdl_trigger();
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
    cov_final_body(tot, f.d, f.P, f.shift_in, (size_t)f.shift_stride, f.shift_f, f.ctl, f.fixed_h, f.target,
                   f.hmin, f.hmax, f.mean_out, f.mean_f_out, f.cov_out, f.L_out);
}


// ----- batched covariance: one launch per stage for many particle sets -----
// A job with tile sums takes them at every iteration (the S phase's gather
// leaves them for iteration 0, the mutation kernel for the later ones);
// otherwise block partials of theta, exactly as the single-run path does.
__global__ void __launch_bounds__(kCovThreads) k_cov_partial_batch(const CovJob* __restrict__ jobs,
                                                                  const int* iter)
{
    const CovJob& j = jobs[blockIdx.y];
    if ((int)blockIdx.x >= j.G || *iter >= j.R || j.tiles) return;
    cov_partial_body(j.theta, j.d, j.P, j.part, blockIdx.x, j.G);
}

__global__ void __launch_bounds__(kCovThreads) k_cov_combine_batch(const CovJob* __restrict__ jobs, const int* iter)
{
    __shared__ double red[32];
    const CovJob& j = jobs[blockIdx.y];
    const int nacc = j.d + j.d * (j.d + 1) / 2;
    const int e = blockIdx.x;
    if (e >= nacc || *iter >= j.R) return;
    const double s = j.tiles ? cov_entry_total<true>(j.tiles, j.ntiles, nacc, e, j.d, j.tile_kd, red)
                                            : cov_entry_total<false>(j.part, j.G, nacc, e, j.d, 0, red);
    if (threadIdx.x == 0) j.part[(size_t)j.G * nacc + e] = s;
}

__global__ void __launch_bounds__(kCovThreads) k_cov_final_batch(const CovJob* __restrict__ jobs, const int* iter)
{
    const CovJob& j = jobs[blockIdx.x];
    if (*iter >= j.R) return;
    const int nacc = j.d + j.d * (j.d + 1) / 2;
    const bool tiles = j.tiles != nullptr;
    cov_final_body(j.part + (size_t)j.G * nacc, j.d, j.P, j.theta, (size_t)j.P, tiles ? j.shift_f : nullptr,
                   j.ctl, 0, j.target, j.hmin, j.hmax, j.mean, j.shift_f, nullptr, j.L);
}

cudaError_t launch_cov_batch(const CovJob* jobs, int n, int Gmax, int dmax, const int* iter, cudaStream_t s)
{
    k_cov_partial_batch<<<dim3(Gmax, n), kCovThreads, 0, s>>>(jobs, iter);
    count_launch();
    k_cov_combine_batch<<<dim3(dmax + dmax * (dmax + 1) / 2, n), kCovThreads, 0, s>>>(jobs, iter);
    count_launch();
    k_cov_final_batch<<<n, kCovThreads, 0, s>>>(jobs, iter);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cov(const double* theta, int d, int P, double* part, int G, unsigned int* counter,
                       Ctl* ctl, int fixed_h_tenths, double acc_target, int hmin, int hmax, double* mean,
                       double* cov, double* L, cudaStream_t s, float* mean_f)
{
    cudaError_t e = pdl_launch(k_cov_partial, dim3(G), dim3(kCovThreads), 0, s, theta, d, P, part);
    count_launch();
    if (e != cudaSuccess) return e;
    const int nacc = d + d * (d + 1) / 2;
    const CovFinalArgs f{d, P, theta, (long long)P, nullptr, ctl, fixed_h_tenths, acc_target, hmin, hmax,
                         mean, mean_f, cov, L, 0};
    e = pdl_launch(k_cov_reduce<false>, dim3(nacc), dim3(kCovThreads), 0, s, (const void*)part, G, nacc,
                   part + (size_t)G * nacc, counter, f);
    count_launch();
    return e;
}

// ----- covariance from the mutation kernel's 32-particle tiles -----
cudaError_t launch_cov_tiles(const float* tiles, int ntiles, int tile_kd, int d, int P, double* tot,
                             unsigned int* counter, float* shift_f, double* mean, Ctl* ctl, int fixed_h_tenths,
                             double acc_target, int hmin, int hmax, double* L, cudaStream_t s)
{
    const int nacc = d + d * (d + 1) / 2;
    const CovFinalArgs f{d, P, nullptr, 1, shift_f, ctl, fixed_h_tenths, acc_target, hmin, hmax, mean,
                         shift_f, nullptr, L, tile_kd};
    const cudaError_t e = pdl_launch(k_cov_reduce<true>, dim3(nacc), dim3(kCovThreads), 0, s,
                                     (const void*)tiles, ntiles, nacc, tot, counter, f);
    count_launch();
    return e;
}

// Independent sampler (Section 3.3): log q of every current particle under
// q = N(qmean, L L'), up to the constant, for the Metropolis-Hastings ratio.
__global__ void __launch_bounds__(256) k_indep_logq(const double* __restrict__ theta, int d, int P,
                                                   const double* __restrict__ L,
                                                   const double* __restrict__ qmean, double* lq)
{
    __shared__ double Ls[kMaxD * kMaxD], ms[kMaxD];
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) Ls[i] = L[i];
    for (int i = threadIdx.x; i < d; i += blockDim.x) ms[i] = qmean[i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const size_t Ps = (size_t)P;
    double u[kMaxD];
    double q = 0.0;
    for (int i = 0; i < d; ++i) {
        double r = theta[i * Ps + p] - ms[i];
        for (int k = 0; k < i; ++k) r -= Ls[i * d + k] * u[k];
        const double piv = Ls[i * d + i];
        u[i] = piv > 0.0 ? r / piv : 0.0;
        q += u[i] * u[i];
    }
    lq[p] = -0.5 * q;
}

cudaError_t launch_indep_logq(const double* theta, int d, int P, const double* L, const double* qmean,
                              double* lq, cudaStream_t s)
{
    k_indep_logq<<<(P + 255) / 256, 256, 0, s>>>(theta, d, P, L, qmean, lq);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adapt_h(Ctl* ctl, int P, double acc_target, int hmin, int hmax, cudaStream_t s)
{
    k_adapt_h<<<1, 32, 0, s>>>(ctl, P, acc_target, hmin, hmax);
    count_launch();
    return cudaGetLastError();
}

// ===================================================== power-tempering search
// RSS(dphi) = (sum_n w_n)^2 / (P sum_n w_n^2) with w_n = exp(dphi (l_n - max l))
// (Section 3.3, pooled over all particles).  One pass evaluates 32 candidate
// increments spread evenly over (lo, hi]: lane c of every warp owns candidate
// c and the warp walks its 32-particle tiles in shared memory.  Candidate
// weights are FP32 hardware exponentials summed in FP32 over one tile (in a
// fixed order); tile sums
// (<= 32) enter 64-bit fixed point (2^-36 units), so block and grid totals are
// exact integer sums whose value does not depend on the order of addition.
// The whole search (max l, then every pass) is one cooperative launch with at
// most one block per SM; blocks meet at bounded grid barriers, and each block
// takes the same decision from the same totals.
constexpr int kSearchThreads = 512;
constexpr int kSearchWarps = kSearchThreads / 32;
constexpr int kCand = 32;
constexpr float kFixScale = 68719476736.0f;       // 2^36

int search_grid(int P)
{
    const int tiles = (P + 31) / 32;
    const int by = (tiles + kSearchWarps - 1) / kSearchWarps;
    const int cap = device_sm_count();
    return by < 1 ? 1 : (by < cap ? by : cap);
}

// Scratch (doubles): 8 barrier words, 3 rotating slots of 64 fixed-point
// totals, one max key per block, then room for the shifted FP32 log
// likelihoods of every tile (used when a block's range exceeds its shared
// memory).
struct SearchScratch {
    unsigned int* bar;            // [0] arrivals, [1] generation, [2] abort
    unsigned long long* acc;      // [3][2 kCand]
    long long* bkey;              // [G]
    float* xf;                    // [P]
};

__host__ __device__ inline SearchScratch search_scratch(double* part, int G)
{
    SearchScratch s;
    s.bar = reinterpret_cast<unsigned int*>(part);
    s.acc = reinterpret_cast<unsigned long long*>(part + 8);
    s.bkey = reinterpret_cast<long long*>(part + 8 + 3 * 2 * kCand);
    s.xf = reinterpret_cast<float*>(part + 8 + 3 * 2 * kCand + G);
    return s;
}

size_t search_part_len(int P)
{
    return 8 + 3 * 2 * kCand + (size_t)search_grid(P) + (size_t)(P + 31) / 32 * 16;
}

size_t search_bar_bytes() { return 8 * sizeof(double); }

// Order-preserving map of a double onto a signed 64-bit key, in integer
// arithmetic (a NaN log likelihood counts as -inf, as in the S phase).
constexpr long long kNegInfBits = (long long)0xfff0000000000000ull;
__device__ __forceinline__ long long order_key(double x)
{
    long long b = __double_as_longlong(x);
    if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) b = kNegInfBits;
    return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
constexpr long long kNegInfKey = kNegInfBits ^ 0x7fffffffffffffffLL;

__device__ __forceinline__ double key_value(long long k)
{
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over the blocks of a cooperative launch.  Arrivals (a release
// add, ordering the block's earlier writes) count up to the grid size; the
// last arrival resets the count and advances the generation (release).  The
// others poll the generation with relaxed loads and take an acquire fence
// once it has moved.  Thread 0 of each block keeps the generation it expects
// to leave (gen, read once before the block's first arrival: the word moves
// only after every block has arrived).  The wait is bounded: every 32 polls it
// checks the abort word and the clock; on time-out (or when another block gave
// up) it sets the abort word and every block returns false.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned int& gen)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned int arrived;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived + 1u == nblocks) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
        } else {
            const uint64_t t0 = global_ns();
            for (unsigned int it = 1; ld_relaxed_u32(bar + 1) == gen; ++it) {
                if ((it & 31u) == 0u && (ld_relaxed_u32(bar + 2) != 0u || global_ns() - t0 > kWaitLimitNs)) {
                    atomicExch(bar + 2, 1u);
                    ok = 0;
                    break;
                }
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
        gen += 1u;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ double candidate(double lo, double hi, int c)
{
    // (c + 1) / kCand as a product with the exact power-of-two reciprocal
    return c == kCand - 1 ? hi : lo + (hi - lo) * ((double)(c + 1) * (1.0 / kCand));
}

__device__ __forceinline__ long long warp_max_key(long long k)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long v = __shfl_xor_sync(0xffffffffu, k, o);
        k = v > k ? v : k;
    }
    return k;
}

// Conversions on the integer pipes.  On this part the FP64 pipe (about two
// lanes per clock per SM) also executes the conversions that touch 64-bit
// values (FP32 <-> 64-bit integer, FP64 <-> FP32), so the search keeps them
// out of its per-particle and per-tile work.
//
// floor(f) for finite f >= 0 (f < 2^64): the 24-bit significand shifted.
__device__ __forceinline__ uint64_t f32_to_u64_floor(float f)
{
    const uint32_t u = __float_as_uint(f);
    if ((u >> 23) == 0u) return 0ull;                 // zero (subnormals are flushed)
    const int e = (int)(u >> 23) - 150;               // f = m 2^e
    const uint64_t m = (uint64_t)((u & 0x7fffffu) | 0x800000u);
    return e >= 0 ? m << e : (e > -24 ? m >> -e : 0ull);
}

// v to FP32 through its two 32-bit halves (each rounded, then one rounded sum).
__device__ __forceinline__ float u64_to_f32(uint64_t v)
{
    return fmaf(__uint2float_rn((uint32_t)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

// d as hi + lo in FP32 from its bits: hi carries the leading 24 significand
// bits (truncated), lo the next 29 (rounded to 24).  ok is false outside
// 2^-126 <= |d| < 2^128 (and for inf or NaN), where the caller converts in FP64.
// The rare FP64 paths of the conversions below, kept out of line so that the
// compiler does not evaluate them speculatively beside the integer path.
__device__ __noinline__ float diff_f64_to_f32(double a, double b) { return __double2float_rn(a - b); }
__device__ __noinline__ float cvt_f64_to_f32(double d) { return __double2float_rn(d); }

__device__ __forceinline__ float2 split_f64(double d, bool& ok)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    ok = e >= -126 && e <= 127;
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
    float lo = 0.0f;
    if (e - 52 >= -126) {
        const float scale = __uint_as_float((uint32_t)(e - 52 + 127) << 23);   // 2^(e - 52)
        lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn((uint32_t)(b & 0x1fffffffu)) * scale));
    }
    return make_float2(hi, lo);
}

// Particles split into one contiguous range of 32-particle tiles per block.
// When a block's range fits (kSearchResident particles) its log likelihoods
// (FP64, read once from HBM) and then their shifted FP32 values stay in its
// shared memory for the whole search; otherwise the FP32 values go to global
// scratch once and every pass stages them, kSearchStage at a time.
constexpr int kSearchResident = 16 * 1024;   // 12 bytes each: 192 KB
constexpr int kSearchStage = 48 * 1024;      // 4 bytes each: 192 KB

size_t search_smem(int P, int G)
{
    const int tpb = ((P + 31) / 32 + G - 1) / G;
    return tpb * 32 <= kSearchResident ? (size_t)tpb * 32 * (sizeof(float) + sizeof(double))
                                       : (size_t)kSearchStage * sizeof(float);
}

__global__ void __launch_bounds__(kSearchThreads, 1) k_power_search(const double* __restrict__ ll, int P,
                                                                   Ctl* ctl, double* part, double d1,
                                                                   int passes)
{
    extern __shared__ __align__(16) float xs[];
    __shared__ long long skey[kSearchWarps];
    __shared__ unsigned long long sacc[2 * kCand];
    __shared__ double scand[kCand];
    __shared__ float sdc[kCand];
    const int G = gridDim.x;
    const SearchScratch sc = search_scratch(part, G);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntiles = (P + 31) / 32;
    const int tpb = (ntiles + G - 1) / G;
    const int t0 = min(ntiles, (int)blockIdx.x * tpb), t1 = min(ntiles, t0 + tpb);
    const int n0 = t0 * 32, nb = (t1 - t0) * 32;   // the block's particles [n0, n0 + nb), padded to tiles
    const bool resident = tpb * 32 <= kSearchResident;
    long long* lraw = reinterpret_cast<long long*>(xs + tpb * 32);   // resident: the FP64 values' bits
    const double phi = ctl->phi;
    unsigned int gen = 0;
    if (threadIdx.x == 0) gen = ld_relaxed_u32(sc.bar + 1);
    if (threadIdx.x < 2 * kCand) sacc[threadIdx.x] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x < 2 * kCand) sc.acc[threadIdx.x] = 0ull;   // slot of pass 0

    // ---- max l over all particles (integer keys: exact, order-free) ----
    long long km = kNegInfKey;
#pragma unroll 4
    for (int i = threadIdx.x; i < nb; i += kSearchThreads) {
        const int n = n0 + i;
        const long long k = n < P ? order_key(ll[n]) : kNegInfKey;
        if (resident) lraw[i] = k;
        km = k > km ? k : km;
    }
    km = warp_max_key(km);
    if (lane == 0) skey[warp] = km;
    __syncthreads();
    if (warp == 0) {
        long long k = lane < kSearchWarps ? skey[lane] : kNegInfKey;
        k = warp_max_key(k);
        if (lane == 0) sc.bkey[blockIdx.x] = k;
    }
    if (!grid_barrier(sc.bar, G, gen)) {
        if (threadIdx.x == 0) raise_error(&ctl->err, kErrTimeout);
        return;
    }
    // every block reads the G block maxima, one per thread (G <= SMs)
    long long kg = (int)threadIdx.x < G ? __ldcg(sc.bkey + threadIdx.x) : kNegInfKey;
    kg = warp_max_key(kg);
    if (lane == 0) skey[warp] = kg;
    __syncthreads();
    kg = warp_max_key(lane < kSearchWarps ? skey[lane] : kNegInfKey);
    const double llmax = key_value(kg);

    // ---- shifted FP32 log likelihoods x_n = l_n - max l (-inf past P) ----
    // (l_hi - max_hi) + (l_lo - max_lo) in FP32: within 2^-23 |x| + 2^-45 |l|.
    bool mok = true;
    const float2 mx = kg == kNegInfKey ? make_float2(0.f, 0.f) : split_f64(llmax, mok);
    // (a resident block converts the keys each thread stored itself)
    float* xdst = resident ? xs : sc.xf + n0;
#pragma unroll 4
    for (int i = threadIdx.x; i < nb; i += kSearchThreads) {
        const int n = n0 + i;
        const long long k = resident ? lraw[i] : (n < P ? order_key(ll[n]) : kNegInfKey);
        float x = -INFINITY;
        if (k != kNegInfKey) {
            const double l = key_value(k);
            bool ok;
            const float2 lx = split_f64(l, ok);
            x = (ok && mok) ? (lx.x - mx.x) + (lx.y - mx.y) : diff_f64_to_f32(l, llmax);
        }
        xdst[i] = x;
    }
    // (the first pass's barrier orders these writes before their reads)

    double lo = 0.0, hi = 1.0 - phi, dphi = hi;
    int done = (kg == kNegInfKey) || !(hi > 0.0);
    int last = done, pass = 0;
    // RSS < D1 compared as (Q1 2^-32)^2 < D1 P 2^4 (Q2 2^-32) in FP32: the
    // fixed-point totals carry 2^-36 units, and FP32 resolves RSS to 1e-7,
    // far inside the error of the FP32 weights themselves.
    const float cmp = (float)(d1 * (double)P * 16.0);
    for (int p = 0; p < passes && !done; ++p) {
        const int slot = p % 3;
        // candidates (FP64) and their FP32 exponent scale, once per block;
        // every candidate is positive (at least (1 - phi) / 32^passes), so
        // dc x is -inf for a dead particle and its weight ex2(-inf) = 0
        if (warp == 0) {
            const double cv = candidate(lo, hi, lane);
            scand[lane] = cv;
            sdc[lane] = fmaxf((float)(cv * kLog2e), 1e-30f);
        }
        __syncthreads();
        const float dc = sdc[lane];
        const float2 dc2 = make_float2(dc, dc);
        unsigned long long q1 = 0ull, q2 = 0ull;
        for (int c0 = 0; c0 < nb; c0 += kSearchStage) {
            const int cn = min(kSearchStage, nb - c0);
            if (!resident) {
                __syncthreads();
                for (int i = threadIdx.x; i < cn; i += kSearchThreads) xs[i] = __ldcg(sc.xf + n0 + c0 + i);
                __syncthreads();
            }
            // lane c owns candidate c; a warp walks its tiles, reading each
            // tile's 32 values as eight broadcast 16-byte loads, two particles
            // per paired FP32 instruction (four partial sums per tile)
            for (int t = warp; t < cn / 32; t += kSearchWarps) {
                const float4* xt = reinterpret_cast<const float4*>(xs + t * 32);
                float2 s1a = make_float2(0.f, 0.f), s1b = s1a, s2a = s1a, s2b = s1a;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 v = xt[u];
                    const float2 ea = __fmul2_rn(dc2, make_float2(v.x, v.y));
                    const float2 eb = __fmul2_rn(dc2, make_float2(v.z, v.w));
                    const float2 wa = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));
                    const float2 wb = make_float2(ex2_approx(eb.x), ex2_approx(eb.y));
                    s1a = __fadd2_rn(s1a, wa);
                    s1b = __fadd2_rn(s1b, wb);
                    s2a = __ffma2_rn(wa, wa, s2a);
                    s2b = __ffma2_rn(wb, wb, s2b);
                }
                const float a1 = (s1a.x + s1a.y) + (s1b.x + s1b.y);
                const float a2 = (s2a.x + s2a.y) + (s2b.x + s2b.y);
                q1 += f32_to_u64_floor(a1 * kFixScale);
                q2 += f32_to_u64_floor(a2 * kFixScale);
            }
        }
        atomicAdd(&sacc[lane], q1);
        atomicAdd(&sacc[kCand + lane], q2);
        __syncthreads();
        if (threadIdx.x < 2 * kCand) {
            atomicAdd(&sc.acc[slot * 2 * kCand + threadIdx.x], sacc[threadIdx.x]);
            sacc[threadIdx.x] = 0ull;
        } else if (blockIdx.x == 0 && threadIdx.x < 4 * kCand) {
            // the slot of the next pass was last read before the previous barrier
            sc.acc[((p + 1) % 3) * 2 * kCand + threadIdx.x - 2 * kCand] = 0ull;
        }
        if (!grid_barrier(sc.bar, G, gen)) {
            if (threadIdx.x == 0) raise_error(&ctl->err, kErrTimeout);
            return;
        }
        // every warp takes the same decision from the same totals
        const float q1s = u64_to_f32(__ldcg(sc.acc + slot * 2 * kCand + lane)) * 2.3283064365386963e-10f;
        const float q2s = u64_to_f32(__ldcg(sc.acc + slot * 2 * kCand + kCand + lane)) * 2.3283064365386963e-10f;
        const unsigned below = __ballot_sync(0xffffffffu, q1s * q1s < cmp * q2s);
        if (below == 0u) {
            // RSS stays >= D1 up to hi: in the first pass this takes the whole
            // remaining power (the last cycle); later it cannot occur because
            // hi was itself a candidate with RSS < D1.
            dphi = hi;
            done = 1;
            last = pass == 0;
        } else {
            const int cc = __ffs(below) - 1;
            const double nlo = cc == 0 ? lo : scand[cc - 1];
            hi = scand[cc];
            lo = nlo;
            dphi = hi;
            pass += 1;
            done = pass >= passes;
            last = 0;
        }
        __syncthreads();   // scand is rewritten by the next pass
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->llmax = llmax;
        ctl->lo = lo;
        ctl->hi = hi;
        ctl->dphi = dphi;
        ctl->pass = pass;
        ctl->done = 1;
        ctl->last = last;
        if (kg == kNegInfKey) raise_error(&ctl->err, kErrDegenerate);
    }
}

// Replay of a recorded power: dphi = phi_l - phi (the rest of the power when
// phi_l = 1), as the C phase of Algorithm 1 with a fixed schedule.
__global__ void k_set_power(Ctl* ctl, double phi_target)
{
    if (threadIdx.x != 0) return;
    const bool last = !(phi_target < 1.0);
    ctl->dphi = last ? 1.0 - ctl->phi : phi_target - ctl->phi;
    ctl->last = last ? 1 : 0;
    ctl->done = 1;
}

cudaError_t launch_set_power(Ctl* ctl, double phi_target, cudaStream_t s)
{
    k_set_power<<<1, 32, 0, s>>>(ctl, phi_target);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_power_search(const double* ll, int P, double d1, int passes, double* part,
                                Ctl* ctl, cudaStream_t s)
{
    int G = search_grid(P);
    const size_t smem = search_smem(P, G);
    static bool attr = false;
    if (!attr) {
        const cudaError_t ea = cudaFuncSetAttribute(k_power_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)(kSearchStage * sizeof(float)));
        if (ea != cudaSuccess) return ea;
        attr = true;
    }
    void* args[] = {(void*)&ll, (void*)&P, (void*)&ctl, (void*)&part, (void*)&d1, (void*)&passes};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_power_search, dim3(G), dim3(kSearchThreads),
                                                      args, smem, s);
    count_launch();
    return e;
}

// ================================================================= S phase
// One block per group.  Weights w_n = exp(log w_n - max_n log w_n), the
// difference formed in FP64 and the exponential in 64-bit fixed point
// (exp_fixed below); log wbar_j(l-1) = max + log(sum_n w_n / N) (Section
// 4.2).  Resampling in integer fixed point (the reading stated in smc.h):
// everything after the quantisation is integer arithmetic, so the selected
// indices do not depend on summation order or thread count.
constexpr int kSelThreads = 1024;

// Shared arrays indexed through sp(n) = n + n/8: a thread's eight
// consecutive entries (the prefix scans give each thread a contiguous range)
// then fall in distinct banks across a warp, 64- and 32-bit alike.
__host__ __device__ __forceinline__ int sp(int n) { return n + (n >> 3); }

size_t select_smem(int N) { return (size_t)sp(N) * (sizeof(uint64_t) + sizeof(uint32_t)); }

__device__ int upper_bound_u64(const uint64_t* a, int n, uint64_t u)
{
    int lo = 0, hi = n;   // first index with a[sp(idx)] > u
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[sp(mid)] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo < n ? lo : n - 1;
}

// Block maximum of 64-bit keys (every thread receives it).
__device__ __forceinline__ long long block_max_key(long long k, long long* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    k = warp_max_key(k);
    __syncthreads();
    if (lane == 0) red[warp] = k;
    __syncthreads();
    k = warp_max_key(lane < (int)(blockDim.x >> 5) ? red[lane] : kNegInfKey);
    return k;
}

// ---- exp(x), x <= 0, in 64-bit fixed point on the integer pipes ----
// The S phase quantises 2^32 exp(x) and sums exp(x) and exp(2x) over the
// group; an FP64 exponential per particle would hold the FP64 pipe (about
// two lanes per clock per SM on this part) for most of the kernel.  Here
// |x| = n ln2/256 + u with 0 <= u < ln2/256, so
//     exp(x) = 2^-(n >> 8) * 2^-((n & 255)/256) * e^-u,
// the middle factor from a table of the 256 powers (units 2^-63, the nearest
// integers) and e^-u from its Taylor polynomial to degree 5, nested as
// 1 - u(1 - u/2(1 - u/3(1 - u/4(1 - u/5)))) (the first omitted term,
// u^6/720 < 2^-60, and each truncation are far below the table's 2^-63).
// |x| enters in units of 2^-57 (exact for |x| >= 2^-5, truncated below);
// ln2/256 in units of 2^-72, so n ln2/256 is exact to 2^-58 for every n here.
// The result M 2^-(63 + k) is within 2^-59 relative of exp(x); |x| >= 64
// (exp(x) < 2^-92, and -inf, NaN) returns false.
__device__ __forceinline__ uint64_t mulq63(uint64_t a, uint64_t b)   // floor(a b / 2^63)
{
    return (__umul64hi(a, b) << 1) | ((a * b) >> 63);
}

__device__ __forceinline__ bool exp_fixed(double x, const uint64_t* tab, uint64_t& M, int& k)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu);
    if (e >= 1029) return false;                                   // |x| >= 64, inf, NaN
    const uint64_t m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
    const int sh = e - 1018;                                       // X = |x| 2^57 < 2^63
    const uint64_t X = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
    constexpr uint64_t kOne = 1ull << 63;
    if (X == 0) {                                                  // |x| < 2^-57: exp(x) rounds to 1
        M = kOne;
        k = 0;
        return true;
    }
    // n = floor(|x| 256/ln2), possibly one too small or too large ...
    long long n = (long long)(__umul64hi(X, kInvLn2x256Q50) >> 43);
    // ... made exact by the sign of the remainder u = |x| - n ln2/256 (2^-72 units)
    __int128 D = ((__int128)X << 15) - (__int128)((unsigned __int128)(uint64_t)n * kLn2Q64);
    if (D < 0) {
        n -= 1;
        D += kLn2Q64;
    } else if (D >= (__int128)kLn2Q64) {
        n += 1;
        D -= kLn2Q64;
    }
    const uint64_t U = (uint64_t)D >> 9;                           // u 2^63 < 2^55
    uint64_t p = kOne - U / 5;
    p = kOne - mulq63(U, p) / 4;
    p = kOne - mulq63(U, p) / 3;
    p = kOne - (mulq63(U, p) >> 1);
    p = kOne - mulq63(U, p);                                       // e^-u 2^63
    M = mulq63(tab[n & 255], p);
    k = (int)(n >> 8);
    return true;
}

// floor(2^32 exp(x)) from the FP64 exponential: out of line, so that the
// compiler does not evaluate it speculatively for every particle.
__device__ __noinline__ uint64_t quantise_fp64_exp(double x) { return (uint64_t)(exp(x) * 4294967296.0); }

// q = floor(2^32 exp(x)) from the fixed-point value, with the group sums'
// terms exp(x) 2^62 and exp(2x) 2^62 (truncated).  When 2^32 exp(x) lies
// within 2^-18 of an integer (the fixed point's error, the FP64 rounding of
// exp(x) and a last-place difference between exponentials all fit well
// inside that), q is taken from the FP64 exponential instead, so that the
// quantised weight is floor(2^32 exp(x)) of the FP64 value exp(x) returns.
__device__ __forceinline__ uint64_t quantise_exp(double x, const uint64_t* tab, uint64_t& w62, uint64_t& w2_62)
{
    uint64_t M;
    int k;
    w62 = w2_62 = 0;
    if (!exp_fixed(x, tab, M, k)) return 0;
    w62 = k < 63 ? M >> (1 + k) : 0ull;
    w2_62 = k < 32 ? __umul64hi(M, M) >> (2 * k) : 0ull;
    const int s = 31 + k;
    if (s >= 64) return 0;                                         // 2^32 exp(x) < 1/2
    const uint64_t q = M >> s;
    const uint64_t rem = M & ((1ull << s) - 1ull);
    const uint64_t mg = 1ull << (s - 18);
    const bool near = (q != 0 && rem < mg) || rem >= (1ull << s) - mg;
    if (M == (1ull << 63) || !near) return q;                        // exp(x) = 1 exactly, or clear of a boundary
    return quantise_fp64_exp(x);
}

// Exact block sums of two 128-bit unsigned values (every thread receives
// them): warp shuffles with carries, then one warp over the warp totals.
__device__ __forceinline__ void add_u128(uint64_t& lo, uint64_t& hi, uint64_t olo, uint64_t ohi)
{
    const uint64_t t = lo + olo;
    hi += ohi + (t < lo ? 1ull : 0ull);
    lo = t;
}

__device__ __forceinline__ void block_sum_u128x2(unsigned __int128& a, unsigned __int128& b, uint64_t* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t v[4] = {(uint64_t)a, (uint64_t)(a >> 64), (uint64_t)b, (uint64_t)(b >> 64)};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
        add_u128(v[0], v[1], w[0], w[1]);
        add_u128(v[2], v[3], w[2], w[3]);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[4 * warp + i] = v[i];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = lane < nw ? red[4 * lane + i] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            uint64_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
            add_u128(v[0], v[1], w[0], w[1]);
            add_u128(v[2], v[3], w[2], w[3]);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) red[i] = v[i];
        }
    }
    __syncthreads();
    a = ((unsigned __int128)red[1] << 64) | red[0];
    b = ((unsigned __int128)red[3] << 64) | red[2];
    __syncthreads();
}

__global__ void __launch_bounds__(kSelThreads) k_select(SelectArgs a)
{
    pdl_trigger();   // the gather may launch and wait while this runs
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int N = a.N;
    double* ws = reinterpret_cast<double*>(sm_raw);                        // w, then q, then prefix r
    uint64_t* qs = reinterpret_cast<uint64_t*>(sm_raw);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(sm_raw + (size_t)sp(N) * sizeof(uint64_t));
    __shared__ long long redk[32];
    __shared__ uint64_t redu[4 * 32];
    __shared__ uint64_t tab[256];
    __shared__ int bad;
    const int j = blockIdx.x;
    const size_t base = (size_t)j * N;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    if (a.mode != 2 && tid < 256) tab[tid] = g_exp2_neg256[tid];

    // ---- weights ----
    // Maxima as order-preserving integer keys and the two weight sums as
    // exact integers: each FP64 instruction holds its pipe for ~64 cycles on
    // this part, so FP64 work per particle is kept to forming log w - max.
    double wmax;
    if (a.mode == 2) {
        long long km = order_key(0.0);
        for (int n = tid; n < N; n += blockDim.x) {
            const double w = a.w[base + n];
            ws[sp(n)] = w;
            const long long k = order_key(w);
            km = k > km ? k : km;
        }
        wmax = key_value(block_max_key(km, redk));
    } else {
        const double dphi = a.mode == 0 ? a.ctl->dphi : 0.0;
        long long km = kNegInfKey;
#pragma unroll 4
        for (int n = tid; n < N; n += blockDim.x) {
            double lw;
            if (a.mode == 0) {
                const double l = a.ll[base + n];
                lw = order_key(l) == kNegInfKey ? -INFINITY : dphi * l;
            } else {
                lw = a.logw[base + n];
            }
            const long long k = order_key(lw);   // NaN counts as -inf
            if (k == kNegInfKey) lw = -INFINITY;
            ws[sp(n)] = lw;
            km = k > km ? k : km;
        }
        const long long kmax = block_max_key(km, redk);   // (its barriers also publish tab)
        const double lmax = key_value(kmax);
        // q_n = floor(2^32 exp(log w_n - max)) straight from the fixed-point
        // exponential, over ws in place; the sums of w and w^2 as exact
        // 128-bit sums of the 2^62-unit terms (order-free), converted once.
        unsigned __int128 S1 = 0, S2 = 0;
        for (int n = tid; n < N; n += blockDim.x) {
            uint64_t q = 0, t1 = 0, t2 = 0;
            if (kmax != kNegInfKey) q = quantise_exp(ws[sp(n)] - lmax, tab, t1, t2);
            qs[sp(n)] = q;
            S1 += t1;
            S2 += t2;
        }
        block_sum_u128x2(S1, S2, redu);
        if (tid == 0) {
            const double s1 = 4.0 * (double)(uint64_t)(S1 >> 64) + 0x1p-62 * (double)(uint64_t)S1;
            const double s2 = 4.0 * (double)(uint64_t)(S2 >> 64) + 0x1p-62 * (double)(uint64_t)S2;
            const double lwj = lmax + log(s1 / (double)N);
            a.lw[j] = lwj;
            a.a[j] += lwj;
            if (a.a_score) a.a_score[j] += lwj;   // log score: cycles after the burn-in
            a.gstat[3 * j + 0] = lmax;
            a.gstat[3 * j + 1] = s1;
            a.gstat[3 * j + 2] = s2;
        }
        wmax = lmax == -INFINITY ? 0.0 : 1.0;
    }
    if (!(wmax > 0.0) || !isfinite(wmax)) {
        if (tid == 0) raise_error(a.err, kErrDegenerate);
        for (int n = tid; n < N; n += blockDim.x) a.idx[base + n] = n;
        return;
    }

    // ---- quantise: q_n = floor(2^32 w_n / max w) ----
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int n0 = min(N, tid * per), n1 = min(N, n0 + per);
    __syncthreads();
    // (From log weights q_n is already in qs.  Given weights: 2^32 w~ is
    // exact, and truncation is the floor of a non-negative number.)
    uint64_t qloc = 0;
    for (int n = n0; n < n1; ++n) {
        if (a.mode == 2) {
            const double w = ws[sp(n)];
            qs[sp(n)] = (uint64_t)((w > 0.0 ? w / wmax : 0.0) * 4294967296.0);
        }
        qloc += qs[sp(n)];
    }
    const uint64_t Q = block_sum<uint64_t>(qloc, redu);
    if (Q == 0) {
        if (tid == 0) raise_error(a.err, kErrDegenerate);
        for (int n = tid; n < N; n += blockDim.x) a.idx[base + n] = n;
        return;
    }
    if (a.scheme >= 2) {
        // Stratified / systematic: slot k takes the particle whose inclusive
        // prefix of q first exceeds floor((k Q + U_k) / N), U_k = mulhi64(x, Q).
        const uint64_t incl = block_inclusive_scan_u64(qloc, redu);
        uint64_t run = incl - qloc;
        for (int n = n0; n < n1; ++n) {
            run += qs[sp(n)];
            qs[sp(n)] = run;
        }
        __syncthreads();
        const bool systematic = a.scheme == 3;
        uint64_t U0 = 0;
        if (systematic) {
            const U64x4 x = philox4x64_10((uint64_t)j, 0, a.cycle, (uint64_t)kTagResample << 32, a.seed, 0);
            U0 = __umul64hi(x.v0, Q);
        }
        for (int k = tid; k < N; k += blockDim.x) {
            uint64_t U = U0;
            if (!systematic) {
                const U64x4 x = philox4x64_10((uint64_t)j, (uint64_t)k, a.cycle, (uint64_t)kTagResample << 32,
                                              a.seed, 0);
                U = __umul64hi(x.v0, Q);
            }
            const uint64_t pos = ((uint64_t)k * Q + U) / (uint64_t)N;
            a.idx[base + k] = upper_bound_u64(qs, N, pos);
        }
        return;
    }
    // ---- deterministic counts and residuals ----
    // floor(N q / Q) from the reciprocal floor((2^64 - 1) / Q): the estimate
    // is the quotient or one less (N q < 2^46), and one step fixes it.
    const uint64_t rQ = ~0ull / Q;
    uint64_t placed = 0, rloc = 0;
    for (int n = n0; n < n1; ++n) {
        const uint64_t q = qs[sp(n)];
        uint64_t c = 0, r = q;
        if (a.scheme == 0) {
            const uint64_t Nq = (uint64_t)N * q;
            c = __umul64hi(Nq, rQ);                    // floor(N w~_n)
            r = Nq - Q * c;
            if (r >= Q) {
                c += 1;
                r -= Q;
            }
        }
        cnt[sp(n)] = (uint32_t)c;
        qs[sp(n)] = r;
        placed += c;
        rloc += r;
    }
    const uint64_t M = (uint64_t)N - block_sum<uint64_t>(placed, redu);
    // inclusive prefix of the residuals
    const uint64_t incl = block_inclusive_scan_u64(rloc, redu);
    uint64_t run = incl - rloc;
    for (int n = n0; n < n1; ++n) {
        run += qs[sp(n)];
        qs[sp(n)] = run;
    }
    __syncthreads();
    const uint64_t R = qs[sp(N - 1)];
    // ---- residual draws ----
    for (uint64_t m = tid; m < M; m += blockDim.x) {
        const U64x4 x = philox4x64_10((uint64_t)j, m, a.cycle, (uint64_t)kTagResample << 32, a.seed, 0);
        const uint64_t u = __umul64hi(x.v0, R);
        const int n = upper_bound_u64(qs, N, u);
        atomicAdd(&cnt[sp(n)], 1u);
    }
    __syncthreads();
    // ---- expand counts into indices ----
    uint64_t cl = 0;
    for (int n = n0; n < n1; ++n) cl += cnt[sp(n)];
    const uint64_t cincl = block_inclusive_scan_u64(cl, redu);
    uint64_t off = cincl - cl;
    for (int n = n0; n < n1; ++n) {
        const uint32_t c = cnt[sp(n)];
        for (uint32_t k = 0; k < c; ++k) {
            if (off < (uint64_t)N) a.idx[base + off] = n;
            else bad = 1;
            ++off;
        }
    }
    __syncthreads();
    if (tid == 0 && bad) raise_error(a.err, kErrBounds);
}

cudaError_t launch_select(const SelectArgs& a, cudaStream_t s)
{
    const size_t sm = select_smem(a.N);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)select_smem(kMaxN));
        attr = true;
    }
    k_select<<<a.J, kSelThreads, sm, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

// The row pointers are staged in shared memory once per block, and each
// thread issues the loads of eight rows before their stores (a plain loop
// waits on every row's load: the compiler cannot tell the rows apart).  With
// kD > 0 the warps then form the covariance tile sums of the particles they
// wrote (cov_tile_sums<kD>, as the mutation kernel's epilogue does).
constexpr int kGatherMaxRows = 2 * kMaxD + 2 + kMaxState;
constexpr int kGatherBatch = 8;

template <int kD>
__global__ void __launch_bounds__(256) k_gather(GatherArgs a)
{
    pdl_trigger();
    __shared__ const double* srow[kGatherMaxRows];
    __shared__ double* drow[kGatherMaxRows];
    __shared__ float shift[kD > 0 ? kD : 1];
    for (int r = threadIdx.x; r < a.nrows; r += blockDim.x) {
        srow[r] = a.src[r];
        drow[r] = a.dst[r];
    }
    pdl_wait();
    __syncthreads();
    if constexpr (kD > 0) {
        if ((int)threadIdx.x < a.d) {
            const float v = (float)srow[threadIdx.x][a.idx[0]];   // slot 0 of group 0
            shift[threadIdx.x] = v;
            if (blockIdx.x == 0) a.covshift[threadIdx.x] = v;
        }
        __syncthreads();
    }
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = s < a.P;
    if (act) {
        const int j = s / a.N;
        const int src = j * a.N + a.idx[s];
        for (int r0 = 0; r0 < a.nrows; r0 += kGatherBatch) {
            double v[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) v[u] = r0 + u < a.nrows ? srow[r0 + u][src] : 0.0;
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u)
                if (r0 + u < a.nrows) drow[r0 + u][s] = v[u];
        }
    }
    if constexpr (kD > 0) cov_tile_sums<kD>(drow[0], (size_t)a.P, a.d, shift, a.covtile, a.ntiles, s, act);
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s)
{
    if (a.nrows < 0 || a.nrows > kGatherMaxRows) return cudaErrorInvalidValue;
    const int kd = a.covtile ? a.tile_kd : 0;
    if (kd > 0 && (a.d < 1 || a.d > kd || !a.covshift || a.nrows < a.d)) return cudaErrorInvalidValue;
    void (*k)(GatherArgs) = nullptr;
    switch (kd) {
    case 0: k = k_gather<0>; break;
    case 5: k = k_gather<5>; break;
    case 8: k = k_gather<8>; break;
    case 11: k = k_gather<11>; break;
    case 14: k = k_gather<14>; break;
    case 17: k = k_gather<17>; break;
    case 20: k = k_gather<20>; break;
    case 23: k = k_gather<23>; break;
    case 26: k = k_gather<26>; break;
    default: return cudaErrorInvalidValue;
    }
    const cudaError_t e = pdl_launch(k, dim3((a.P + 255) / 256), dim3(256), 0, s, a);
    count_launch();
    return e;
}

// Double-float accumulation on the FP32 pipe (Knuth's TwoSum): x + b and x + y.
__device__ __forceinline__ Df df_add_f(Df x, float b)
{
    const float s = x.hi + b;
    const float bv = s - x.hi;
    const float e = (x.hi - (s - bv)) + (b - bv);
    return df_quick(s, e + x.lo);
}

__device__ __forceinline__ Df df_add(Df x, Df y)
{
    const float s = x.hi + y.hi;
    const float bv = s - x.hi;
    const float e = (x.hi - (s - bv)) + (y.hi - bv);
    return df_quick(s, e + (x.lo + y.lo));
}

__device__ __forceinline__ Df warp_sum_df(Df x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Df y = {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
        x = df_add(x, y);
    }
    return x;
}

// FP64 -> FP32, round to nearest even, from the bits (the conversion
// instruction for values outside the normal FP32 range).
__device__ __forceinline__ float f64_to_f32(double d)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
    if (e - 897u >= 254u) return cvt_f64_to_f32(d);          // FP32 exponent outside 1..254
    const uint64_t mant = b & 0xfffffffffffffull;
    uint32_t f = ((uint32_t)(b >> 32) & 0x80000000u) | ((e - 896u) << 23) | (uint32_t)(mant >> 29);
    const uint32_t rest = (uint32_t)mant & 0x1fffffffu;          // the 29 bits rounded away
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;   // carries into the exponent
    return __uint_as_float(f);
}

// Data-tempering stop search of one chunk (Section 3.3, "C phase
// termination"): block q combines the G blocks' (max log w, sum w, sum w^2)
// of observation s0 + q + 1 into the pooled RSS; the last block to finish
// takes the first observation with RSS < D1 (or a date of interest, or T) as
// the end of the chunk.  The block maxima are compared as order-preserving
// integer keys; the rescaling weights exp(M_g - M) are FP32 exponentials of
// the differences formed from the FP32 hi/lo splits of the FP64 values (the
// blocks' sums are themselves sums of FP32 weights, ~1e-7), accumulated as
// double-float pairs on the FP32 pipe, with no FP64 instruction per block
// and observation.  (One warp doing it all in FP64 took ~0.5 ms per chunk at
// 512 blocks: each FP64 instruction holds this part's FP64 pipe for ~64
// cycles; one warp per observation in a single block, 39 us per chunk at
// 293 blocks.)  The per-observation results and the arrival count sit in a
// tail of the chunk scratch (cdata_part_len); the count returns to zero.
constexpr int kCdSelThreads = 32 * kCdataChunk;   // k_pit_final: one warp per observation
constexpr int kCdStopThreads = 256;

size_t cdata_part_len(int G) { return (size_t)G * kCdataChunk * 3 + 2 * kCdataChunk + 8; }

struct CdStopTail {
    double* rss;           // [kCdataChunk]
    int* flag;             // [kCdataChunk]
    unsigned int* count;   // arrivals of the current launch
};

__device__ __forceinline__ CdStopTail cdstop_tail(double* part, int G)
{
    double* t = part + (size_t)G * kCdataChunk * 3;
    return {t, reinterpret_cast<int*>(t + kCdataChunk), reinterpret_cast<unsigned int*>(t + 2 * kCdataChunk)};
}

__global__ void __launch_bounds__(kCdStopThreads) k_cdata_select(double* part, int G, int B, int s0, int T, int P,
                                                                double d1, ForceDates fd, Ctl* ctl, int seq)
{
    constexpr int kW = kCdStopThreads / 32;
    __shared__ long long sk[kW];
    __shared__ float sd[4][kW];
    __shared__ int last;
    if (ctl->cd_found != 0) return;   // an earlier chunk of this cycle holds the stop
    const int q = blockIdx.x;   // gridDim.x = B
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const CdStopTail tl = cdstop_tail(part, G);
    long long km = kNegInfKey;
    for (int g = tid; g < G; g += kCdStopThreads) {
        const long long k = order_key(part[((size_t)g * B + q) * 3]);
        km = k > km ? k : km;
    }
    km = warp_max_key(km);
    if (lane == 0) sk[w] = km;
    __syncthreads();
    km = warp_max_key(lane < kW ? sk[lane] : kNegInfKey);
    Df s1 = {0.0f, 0.0f}, s2 = {0.0f, 0.0f};
    if (km != kNegInfKey) {
        bool mok;
        const float2 mx = split_f64(key_value(km), mok);
        const double M = key_value(km);
        for (int g = tid; g < G; g += kCdStopThreads) {
            const double* o = part + ((size_t)g * B + q) * 3;
            if (order_key(o[0]) == kNegInfKey) continue;
            bool ok;
            const float2 ox = split_f64(o[0], ok);
            const float x = (ok && mok) ? (ox.x - mx.x) + (ox.y - mx.y) : diff_f64_to_f32(o[0], M);
            const float e = ex2_approx(x * (float)kLog2e);
            s1 = df_add_f(s1, f64_to_f32(o[1]) * e);
            s2 = df_add_f(s2, f64_to_f32(o[2]) * (e * e));
        }
    }
    s1 = warp_sum_df(s1);
    s2 = warp_sum_df(s2);
    if (lane == 0) {
        sd[0][w] = s1.hi;
        sd[1][w] = s1.lo;
        sd[2][w] = s2.hi;
        sd[3][w] = s2.lo;
    }
    __syncthreads();
    if (tid == 0) {
        Df a = {0.0f, 0.0f}, b = {0.0f, 0.0f};
        for (int i = 0; i < kW; ++i) {   // fixed order
            a = df_add(a, Df{sd[0][i], sd[1][i]});
            b = df_add(b, Df{sd[2][i], sd[3][i]});
        }
        const double S1 = (double)a.hi + (double)a.lo, S2 = (double)b.hi + (double)b.lo;
        const double rss = S1 * S1 / ((double)P * S2);
        const int sobs = s0 + q + 1;
        bool date = sobs == T;
        for (int i = 0; i < fd.n; ++i) date = date || fd.t[i] == sobs;
        const bool low = !(rss >= d1);   // RSS < D1 (a degenerate NaN also stops)
        tl.rss[q] = rss;
        tl.flag[q] = ((low || date) ? 1 : 0) | ((date && !low) ? 2 : 0);
        __threadfence();
        last = atomicAdd(tl.count, 1u) == (unsigned int)B - 1u;
    }
    __syncthreads();
    if (!last || tid >= 32) return;
    __threadfence();
    const int f = tid < B ? __ldcg(tl.flag + tid) : 0;
    const unsigned m = __ballot_sync(0xffffffffu, (f & 1) != 0);
    const int at = m ? __ffs(m) - 1 : (B - 1);
    if (tid == 0) {
        ctl->cd_stop = m ? at + 1 : B;
        ctl->cd_found = m ? seq : 0;
        ctl->cd_forced = m ? (__ldcg(tl.flag + at) >> 1) & 1 : 0;
        ctl->rss = __ldcg(tl.rss + at);
        *tl.count = 0u;
    }
}

// PIT of the committed observations s0 + 1 .. s0 + stop (Section 4.1): warp q
// combines the blocks' (max log w(s-1), sum w, sum w I[Y_s <= y_s]) of
// observation s0 + q + 1 into the weighted share (FP64 throughout: the PIT is
// compared with the oracle's to 1e-9).
__global__ void __launch_bounds__(kCdSelThreads) k_pit_final(const double* part, int G, int B, int s0,
                                                            const Ctl* ctl, double* pit, int seq)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int found = ctl->cd_found;
    if ((found != 0 && found < seq) || q >= ctl->cd_stop || q >= B) return;
    long long km = kNegInfKey;
    for (int g = lane; g < G; g += 32) {
        const long long k = order_key(part[((size_t)g * B + q) * 3]);
        km = k > km ? k : km;
    }
    km = warp_max_key(km);
    const double M = key_value(km);
    double S1 = 0.0, S2 = 0.0;
    if (km != kNegInfKey)
        for (int g = lane; g < G; g += 32) {
            const double* o = part + ((size_t)g * B + q) * 3;
            if (order_key(o[0]) == kNegInfKey) continue;
            const double e = exp(o[0] - M);
            S1 += o[1] * e;
            S2 += o[2] * e;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S1 += __shfl_xor_sync(0xffffffffu, S1, o);
        S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    }
    if (lane == 0) pit[s0 + q] = S2 / S1;
}

cudaError_t launch_pit_final(const double* part, int G, int B, int s0, const Ctl* ctl, double* pit, int seq,
                             cudaStream_t s)
{
    k_pit_final<<<1, kCdSelThreads, 0, s>>>(part, G, B, s0, ctl, pit, seq);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cdata_select(double* part, int G, int B, int s0, int T, int P, double d1,
                                const ForceDates& fd, Ctl* ctl, int seq, cudaStream_t s)
{
    k_cdata_select<<<B, kCdStopThreads, 0, s>>>(part, G, B, s0, T, P, d1, fd, ctl, seq);
    count_launch();
    return cudaGetLastError();
}

// Pooled RSS at the chosen power from per-group (max, sum, sum of squares),
// log wtilde += log(J^-1 sum_j wbar_j(l-1)), and phi += dphi.
// Four warps: warps 0-1 pool the groups' (max, sum w, sum w^2) into the RSS,
// warps 2-3 the groups' log w-bar into log w-tilde; maxima as integer keys,
// and the closing arithmetic split over three threads of different warps
// (each FP64 instruction holds its scheduler's pipe for ~64 cycles).
__global__ void __launch_bounds__(128) k_cycle_close(const double* gstat, const double* lw, int J, int N, int power,
                                                     Ctl* ctl)
{
    pdl_trigger();
    pdl_wait();
    __shared__ long long sk[4];
    __shared__ double sa[4], sb[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool pool = warp < 2;   // else: log w-tilde
    const int t = tid & 63;
    long long km = kNegInfKey;
    for (int j = t; j < J; j += 64) {
        const long long k = order_key(pool ? gstat[3 * j] : lw[j]);
        km = k > km ? k : km;
    }
    km = warp_max_key(km);
    if (lane == 0) sk[warp] = km;
    __syncthreads();
    const long long k0 = sk[pool ? 0 : 2], k1 = sk[pool ? 1 : 3];
    const long long kmax = k0 > k1 ? k0 : k1;
    const double mx = key_value(kmax);
    double a = 0.0, b = 0.0;
    if (kmax != kNegInfKey)
        for (int j = t; j < J; j += 64) {
            if (pool) {
                const double m = gstat[3 * j];
                if (order_key(m) == kNegInfKey) continue;
                const double e = exp(m - mx);
                a += gstat[3 * j + 1] * e;
                b += gstat[3 * j + 2] * e * e;
            } else {
                a += exp(lw[j] - mx);
            }
        }
    a = warp_sum(a);
    if (pool) b = warp_sum(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (tid == 0) {
        const double s1 = sa[0] + sa[1], s2 = sb[0] + sb[1];
        ctl->rss = s1 * s1 / ((double)J * (double)N * s2);
    } else if (tid == 64) {
        ctl->ltilde += mx + log((sa[2] + sa[3]) / (double)J);
    } else if (tid == 32) {
        if (power) ctl->phi = ctl->last ? 1.0 : ctl->phi + ctl->dphi;
        ctl->acc_sum = 0.0;
        ctl->acc_n = 0;
    }
}

cudaError_t launch_cycle_close(const double* gstat, const double* lw, int J, int N, int power,
                               Ctl* ctl, cudaStream_t s)
{
    const cudaError_t e = pdl_launch(k_cycle_close, dim3(1), dim3(128), 0, s, gstat, lw, J, N, power, ctl);
    count_launch();
    return e;
}

// ===================================================== moments and estimators
// Test functions of Section 5.2 at the end state (v_kt, eps_t).
template <typename Real, int K, int I>
__global__ void k_testfn(ModelDev m, const double* __restrict__ theta, const double* __restrict__ state,
                         int P, double* g)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const size_t Ps = (size_t)P;
    double th[kMaxD];
    for (int i = 0; i < m.d; ++i) th[i] = theta[i * Ps + p];
    Real full[kMaxD];
    full_theta<Real>(m, th, full);
    EgarchParams<Real, K, I> q;
    egarch_transform<Real, K, I>(full, m.gamma, q);
    const Real eps = (Real)state[K * Ps + p];
    Real vs = 0, vn = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const Real v = (Real)state[k * Ps + p];
        vs += v;
        vn += q.alpha[k] * v + q.beta[k] * (fabs(eps) - (Real)kSqrt2OverPi) + q.gamma[k] * eps;
    }
    const Real g1 = q.log_sigma_y + vs / Real(2);
    Real g2 = 0;
#pragma unroll
    for (int i = 0; i < I; ++i) g2 += q.p[i] * (q.mu[i] * q.mu[i] * q.mu[i] + Real(3) * q.mu[i] * q.sig[i] * q.sig[i]);
    const Real hn = exp(q.log_sigma_y + vn / Real(2));
    const Real x = (Real(-0.03) - q.mu_y) / hn;
    Real g3 = 0;
#pragma unroll
    for (int i = 0; i < I; ++i) g3 += q.p[i] * Real(0.5) * erfc(-((x - q.mu[i]) / q.sig[i]) * (Real)0.70710678118654752440);
    g[0 * Ps + p] = (double)g1;
    g[1 * Ps + p] = (double)g2;
    g[2 * Ps + p] = (double)g3;
}

template <typename Real, int K>
static void testfn_k(const ModelDev& m, const double* th, const double* st, int P, double* g, cudaStream_t s)
{
    const int G = (P + 255) / 256;
    switch (m.I) {
    case 1: k_testfn<Real, K, 1><<<G, 256, 0, s>>>(m, th, st, P, g); break;
    case 2: k_testfn<Real, K, 2><<<G, 256, 0, s>>>(m, th, st, P, g); break;
    case 3: k_testfn<Real, K, 3><<<G, 256, 0, s>>>(m, th, st, P, g); break;
    default: k_testfn<Real, K, 4><<<G, 256, 0, s>>>(m, th, st, P, g); break;
    }
}

template <typename Real>
static void testfn_real(const ModelDev& m, const double* th, const double* st, int P, double* g, cudaStream_t s)
{
    switch (m.K) {
    case 1: testfn_k<Real, 1>(m, th, st, P, g, s); break;
    case 2: testfn_k<Real, 2>(m, th, st, P, g, s); break;
    case 3: testfn_k<Real, 3>(m, th, st, P, g, s); break;
    default: testfn_k<Real, 4>(m, th, st, P, g, s); break;
    }
}

cudaError_t launch_testfn(const ModelDev& m, int precision, const double* theta,
                          const double* state, int P, double* g, cudaStream_t s)
{
    if (precision == 1) testfn_real<float>(m, theta, state, P, g, s);
    else testfn_real<double>(m, theta, state, P, g, s);
    count_launch();
    return cudaGetLastError();
}

// Per group and function: mean and centred sum of squares (two passes in the
// block), combined across groups with the parallel formula
//   sum_jn (g - gbar)^2 = sum_j [M2_j + N (gbar_j - gbar)^2].
__global__ void k_group_moments(const double* __restrict__ g, int nf, int N, int P, double* part)
{
    __shared__ double red[32];
    const int j = blockIdx.x, f = blockIdx.y;
    const double* row = g + (size_t)f * P + (size_t)j * N;
    double s = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) s += row[n];
    const double mean = block_sum(s, red) / (double)N;
    double q = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double e = row[n] - mean;
        q += e * e;
    }
    q = block_sum(q, red);
    if (threadIdx.x == 0) {
        part[((size_t)f * gridDim.x + j) * 2 + 0] = mean;
        part[((size_t)f * gridDim.x + j) * 2 + 1] = q;
    }
}

__global__ void k_moments_final(const double* part, int nf, int J, int N, double* out, Ctl* ctl,
                                int rne_from)
{
    __shared__ double rne_s[64];
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        const double* pf = part + (size_t)f * J * 2;
        double gbar = 0.0;
        for (int j = 0; j < J; ++j) gbar += pf[2 * j];
        gbar /= (double)J;                                   // (garnd_approx)
        double between = 0.0, within = 0.0;
        for (int j = 0; j < J; ++j) {
            const double e = pf[2 * j] - gbar;
            between += e * e;
            within += pf[2 * j + 1];
        }
        const double total = within + (double)N * between;
        const double var_hat = total / ((double)N * J - 1.0);
        const double v_hat = (double)N / (J - 1.0) * between;    // (vhat)
        out[4 * f + 0] = gbar;
        out[4 * f + 1] = sqrt(var_hat);
        out[4 * f + 2] = sqrt(between / ((double)J * (J - 1.0)));  // (NSE_def)
        out[4 * f + 3] = v_hat > 0.0 ? var_hat / v_hat : INFINITY;
        if (f < 64) rne_s[f] = out[4 * f + 3];
    }
    __syncthreads();
    if (ctl && threadIdx.x == 0) {
        double s = 0.0;
        int n = 0;
        for (int f = rne_from; f < nf && f < 64; ++f) {
            s += rne_s[f];
            ++n;
        }
        ctl->mean_rne = n ? s / n : 0.0;
    }
}

cudaError_t launch_moments(const double* g, int nf, int J, int N, double* part, double* out,
                           Ctl* ctl, int rne_from, cudaStream_t s)
{
    dim3 grid(J, nf);
    k_group_moments<<<grid, 256, 0, s>>>(g, nf, N, J * N, part);
    count_launch();
    k_moments_final<<<1, 64, 0, s>>>(part, nf, J, N, out, ctl, rne_from);
    count_launch();
    return cudaGetLastError();
}

// log wbar = log J^-1 sum_j exp(a_j); NSE of log wbar from (ML_se):
// [J (J-1)]^-1 sum_j (wbar_j - wbar)^2 / wbar^2, all scaled by exp(max a).
__global__ void k_ml(const double* a, int J, const Ctl* ctl, double* out)
{
    const int lane = threadIdx.x;
    double amax = -INFINITY;
    for (int j = lane; j < J; j += 32) amax = fmax(amax, a[j]);
    amax = warp_max(amax);
    double rs = 0.0;
    for (int j = lane; j < J; j += 32) rs += exp(a[j] - amax);
    const double rbar = warp_sum(rs) / (double)J;
    double ss = 0.0;
    for (int j = lane; j < J; j += 32) {
        const double r = exp(a[j] - amax) - rbar;
        ss += r * r;
    }
    ss = warp_sum(ss);
    if (lane != 0) return;
    out[0] = amax + log(rbar);
    out[1] = sqrt(ss / ((double)J * (J - 1.0))) / rbar;
    out[2] = ctl ? ctl->ltilde : 0.0;
}

cudaError_t launch_ml(const double* a, int J, const Ctl* ctl, double* out, cudaStream_t s)
{
    k_ml<<<1, 32, 0, s>>>(a, J, ctl, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace smc
