// Per-particle likelihood recursions and the observation pipeline.
//
// EGARCH(K, I) of Section 5.1: parameters from Table 1 through the transforms
// (EGARCH_tran1)-(EGARCH_tran2); for t = 1..T
//   v_kt  = alpha_k v_k,t-1 + beta_k (|eps_t-1| - (2/pi)^1/2) + gamma_k eps_t-1
//   h_t   = sigma_Y exp(sum_k v_kt / 2),   eps_t = (y_t - mu_Y) / h_t
//   l_t   = -1/2 log 2pi - log h_t + log sum_i p_i / sigma_i exp(-(eps_t - mu_i)^2 / 2 sigma_i^2)
// with v_k0 = 0 and no shock before the first observation (v_k1 = 0; the
// eps_0 = 0 reading v_k1 = -beta_k (2/pi)^1/2 is selectable).
//
// FP32 path (EgarchF32): the recursion runs in base-2 units so that every
// exponential is one hardware ex2:
//   v'_k = v_k log2(e) / 2, eps scaled by s = (log2(e)/2)^1/2,
//   log2 h_t = log2 sigma_Y + sum_k v'_kt,
//   mixture exponent x_it = log2(p_i / sigma_i) - (s (eps_t - mu_i) / sigma_i)^2.
// The mixture log-sum-exp is max-shifted; the shifted sums s_t in [1, I] are
// multiplied together and one lg2 is taken per 32 observations.  Sums of the
// per-observation terms stay in FP32 for 256 observations and are then added
// into an FP64 accumulator (the log likelihood itself is FP64).
// FP64 path (EgarchF64): the four steps as written, in double precision.
#pragma once

#include "common.cuh"

namespace smc {

constexpr double kLog2Pi = 1.83787706640934548356;
constexpr double kSqrt2OverPi = 0.79788456080286535588;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;
constexpr double kSfac = 0.84932180028801904272;       // (log2(e) / 2)^1/2
constexpr double kLog2Sfac = -0.23561681352755119288;  // log2 of kSfac
constexpr double kLogSfac = -0.16331712998914049120;   // ln of kSfac

// Device view of a model, passed by value in kernel parameters so that every
// thread reads it through the uniform constant path.
struct ModelDev {
    int kind;        // 0 EGARCH, 1 LINREG
    int K, I, gamma, eps0_zero;
    int p;           // LINREG regressors
    double sigma;    // LINREG disturbance s.d.
    int d_full, d;
    int has_free;    // 0: all d_full parameters free
    int free_idx[kMaxD];
    double theta_fixed[kMaxD];
    double prior_mean[kMaxD];
    double prior_isd[kMaxD];   // 1 / prior s.d.
    double prior_c[kMaxD];     // -1/2 log 2pi - log prior s.d.
    double prior_lo[kMaxD];
    // the same prior constants rounded to FP32 (FP32 log prior)
    float prior_mean_f[kMaxD], prior_isd_f[kMaxD], prior_c_f[kMaxD], prior_lo_f[kMaxD];
};

// Full parameter vector from a particle's free parameters.
template <typename Real>
__device__ __forceinline__ void full_theta(const ModelDev& m, const double* th, Real* full)
{
    if (!m.has_free) {
        for (int i = 0; i < m.d_full; ++i) full[i] = (Real)th[i];
        return;
    }
    for (int i = 0; i < m.d_full; ++i) full[i] = (Real)m.theta_fixed[i];
    for (int k = 0; k < m.d; ++k) full[m.free_idx[k]] = (Real)th[k];
}

// Full parameter vector from FP32 free parameters.
__device__ __forceinline__ void full_theta_f(const ModelDev& m, const float* th, float* full)
{
    if (!m.has_free) {
        for (int i = 0; i < m.d_full; ++i) full[i] = th[i];
        return;
    }
    for (int i = 0; i < m.d_full; ++i) full[i] = (float)m.theta_fixed[i];
    for (int k = 0; k < m.d; ++k) full[m.free_idx[k]] = th[k];
}

// The log prior in FP32 arithmetic on thf = (float)th (the FP32 path, whose
// likelihood carries FP32 error far above it).  The support test is exact:
// rounding is monotone, so thf > (float)lo implies th >= lo, and otherwise th
// itself is compared in FP64.
__device__ __forceinline__ double log_prior_f(const ModelDev& m, const double* th, const float* thf)
{
    float lp = 0.0f;
    for (int k = 0; k < m.d; ++k) {
        const float x = thf[k];
        if (!(x > m.prior_lo_f[k]) && !(th[k] >= m.prior_lo[k])) return -INFINITY;
        if (!isfinite(x)) return -INFINITY;
        const float z = (x - m.prior_mean_f[k]) * m.prior_isd_f[k];
        lp += m.prior_c_f[k] - 0.5f * z * z;
    }
    return (double)lp;
}

// Log prior density kernel (Gaussian per free parameter, truncated below).
__device__ __forceinline__ double log_prior(const ModelDev& m, const double* th)
{
    double lp = 0.0;
    for (int k = 0; k < m.d; ++k) {
        const double x = th[k];
        if (!(x >= m.prior_lo[k]) || !isfinite(x)) return -INFINITY;
        const double z = (x - m.prior_mean[k]) * m.prior_isd[k];
        lp += m.prior_c[k] - 0.5 * z * z;
    }
    return lp;
}

// Table 1 transforms and (EGARCH_tran1)-(EGARCH_tran2).
template <typename Real, int K, int I>
struct EgarchParams {
    Real mu_y, log_sigma_y;
    Real alpha[K], beta[K], gamma[K];
    Real p[I], mu[I], sig[I];
};

template <typename Real, int K, int I>
__device__ __forceinline__ void egarch_transform(const Real* th, int has_gamma,
                                                 EgarchParams<Real, K, I>& q)
{
    int j = 0;
    q.mu_y = th[j++] / Real(1000);
    q.log_sigma_y = th[j++];
#pragma unroll
    for (int k = 0; k < K; ++k) q.alpha[k] = tanh(th[j + k]);
    j += K;
#pragma unroll
    for (int k = 0; k < K; ++k) q.beta[k] = exp(th[j + k]);
    j += K;
#pragma unroll
    for (int k = 0; k < K; ++k) q.gamma[k] = has_gamma ? th[j + k] : Real(0);
    if (has_gamma) j += K;
    if constexpr (I == 1) {
        q.p[0] = Real(1);
        q.mu[0] = Real(0);
        q.sig[0] = Real(1);
    } else {
        Real pstar[I], mustar[I], sigstar[I];
#pragma unroll
        for (int i = 0; i < I; ++i) pstar[i] = Real(2) / (Real(1) + exp(Real(-2) * th[j + i]));  // tanh + 1 without cancellation
#pragma unroll
        for (int i = 0; i < I; ++i) mustar[i] = th[j + I + i];
#pragma unroll
        for (int i = 0; i < I; ++i) sigstar[i] = exp(th[j + 2 * I + i]);
        Real psum = 0;
#pragma unroll
        for (int i = 0; i < I; ++i) psum += pstar[i];
        Real pmu = 0;
#pragma unroll
        for (int i = 0; i < I; ++i) {
            q.p[i] = pstar[i] / psum;
            pmu += q.p[i] * mustar[i];
        }
        Real s = 0;
        Real mu2[I];
#pragma unroll
        for (int i = 0; i < I; ++i) {
            mu2[i] = mustar[i] - pmu;
            s += q.p[i] * (mu2[i] * mu2[i] + sigstar[i] * sigstar[i]);
        }
        const Real c = Real(1) / sqrt(s);
#pragma unroll
        for (int i = 0; i < I; ++i) {
            q.mu[i] = c * mu2[i];
            q.sig[i] = c * sigstar[i];
        }
    }
}

// ------------------------------------------------------------- FP32 recursion
// The first factor carries log2 sigma_Y - log2 s: u = lsy2p + v'_1, so that
// log2 h - log2 s = u + v'_2 + ... + v'_K; its update is
//   u_t = alpha_1 u_t-1 + (1 - alpha_1) lsy2p + beta'_1 |es| + gamma'_1 es - beta_1 c log2(e)/2.
// Each update is split into alpha v + const (independent of the last shock,
// so it overlaps the previous exponential) and the shock terms, which keeps
// the per-observation dependency chain to two FMAs, one add, one ex2 and one
// multiply.
//
// kDelta (the stand-alone likelihood and the data-tempering C phase, which
// see raw prior draws): alpha_k = tanh(theta_3k) close to 1 loses most of
// 1 - alpha_k when rounded to FP32 (its ulp is 6e-8, so 1 - alpha = 1e-3 keeps
// only ~4 digits), and the recursion's long memory 1 / (1 - alpha) turns that
// into a systematic error of the volatility level.  This form carries
// delta_k = 1 - alpha_k = 2 / (1 + e^(2 theta_3k)), formed directly in FP32
// (relative error ~1e-7), and updates alpha v as v - delta v (one FMA, single
// rounding); lsy2p then stays out of the first factor and enters log2 h as
// its own term.  Two more FP32 operations per observation.
template <int K, int I, bool kDelta = false>
struct EgarchF32 {
    float mu, lsy2p;                       // mu_Y; log2 sigma_Y - log2 s
    float al[K], be[K], ga[K], nb[K];      // alpha (kDelta: 1 - alpha); beta, gamma in scaled units; constant term
    float a[I], b[I], c[I];                // 1/sigma_i; -mu_i s / sigma_i; log2(p_i / sigma_i)
    float v0[K];                           // state after the first observation's update
    float v[K], es;                        // recursion state (scaled units; v[0] includes lsy2p)
    float sh, sm, prod;                    // partial sums over the current 32 observations
    float part;                            // sum of the completed 32-observation partials (<= 256 obs)
    double acc;                            // FP64 sum of completed partials (log2 units)

    __device__ __forceinline__ void setup(const float* th, int has_gamma, int eps0_zero)
    {
        EgarchParams<float, K, I> q;
        egarch_transform<float, K, I>(th, has_gamma, q);
        mu = q.mu_y;
        lsy2p = q.log_sigma_y * (float)kLog2e - (float)kLog2Sfac;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            // theta_3k sits at index 2 + k (Table 1 order)
            al[k] = kDelta ? 2.0f / (1.0f + expf(2.0f * th[2 + k])) : q.alpha[k];
            be[k] = q.beta[k] * (float)(kLog2e / 2.0 / kSfac);
            ga[k] = q.gamma[k] * (float)(kLog2e / 2.0 / kSfac);
            const float c0 = -q.beta[k] * (float)(kSqrt2OverPi * kLog2e / 2.0);
            nb[k] = c0;
            v0[k] = eps0_zero ? c0 : 0.0f;
        }
        if constexpr (!kDelta) {
            nb[0] = fmaf(1.0f - al[0], lsy2p, nb[0]);
            v0[0] += lsy2p;
        }
#pragma unroll
        for (int i = 0; i < I; ++i) {
            a[i] = 1.0f / q.sig[i];
            b[i] = -q.mu[i] * (float)kSfac / q.sig[i];
            c[i] = log2f(q.p[i] / q.sig[i]);
        }
        es = 0.0f;
        sh = sm = 0.0f;
        prod = 1.0f;
        part = 0.0f;
        acc = 0.0;
    }

    __device__ __forceinline__ void update_volatility_first()
    {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = v0[k];
    }

    __device__ __forceinline__ void update_volatility()
    {
        float vp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if constexpr (kDelta) vp[k] = fmaf(-al[k], v[k], v[k]) + nb[k];
            else vp[k] = fmaf(al[k], v[k], nb[k]);
        }
        const float ae = fabsf(es);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = fmaf(be[k], ae, fmaf(ga[k], es, vp[k]));
    }

    // e = log2 h_t - log2 s
    __device__ __forceinline__ float log2h() const
    {
        float e = kDelta ? lsy2p + v[0] : v[0];
#pragma unroll
        for (int k = 1; k < K; ++k) e += v[k];
        return e;
    }

    // The volatility part of one observation (log2 h, its sum, the shock):
    // step = chain + mix.
    template <bool kFirst>
    __device__ __forceinline__ void chain(float y)
    {
        if constexpr (kFirst) update_volatility_first();
        else update_volatility();
        const float e = log2h();
        sh += e;
        es = (y - mu) * ex2_approx(-e);
    }

    // The mixture part of one observation for the shock x (scaled units).
    __device__ __forceinline__ void mix(float x)
    {
        if constexpr (I == 1) {
            sm = fmaf(-x, x, sm);
        } else if constexpr (I == 2) {
            const float z0 = fmaf(a[0], x, b[0]), z1 = fmaf(a[1], x, b[1]);
            const float x0 = fmaf(-z0, z0, c[0]), x1 = fmaf(-z1, z1, c[1]);
            sm += fmaxf(x0, x1);
            prod = fmaf(prod, ex2_approx(-fabsf(x0 - x1)), prod);
        } else {
            float xs[I];
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const float z = fmaf(a[i], x, b[i]);
                xs[i] = fmaf(-z, z, c[i]);
            }
            float m = xs[0];
#pragma unroll
            for (int i = 1; i < I; ++i) m = fmaxf(m, xs[i]);
            float s = ex2_approx(xs[0] - m);
#pragma unroll
            for (int i = 1; i < I; ++i) s += ex2_approx(xs[i] - m);
            sm += m;
            prod *= s;
        }
    }

    template <bool kFirst>
    __device__ __forceinline__ void step(float y)
    {
        chain<kFirst>(y);
        mix(es);
    }

    // Continue from a saved state (natural units) and evaluate one observation's
    // log density l_t in natural units (data-tempering C phase).
    __device__ __forceinline__ void load_state(const double* st)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = (float)(st[k] * (kLog2e / 2.0));
        if constexpr (!kDelta) v[0] += lsy2p;
        es = (float)(st[K] * kSfac);
    }

    // One observation's log density less the constant kTermConst, in log2
    // units: l_t = ln2 u + kTermConst.
    template <bool kFirst>
    __device__ __forceinline__ float logdens2(float y)
    {
        if constexpr (kFirst) update_volatility_first();
        else update_volatility();
        const float e = log2h();
        es = (y - mu) * ex2_approx(-e);
        float u;
        if constexpr (I == 1) {
            u = fmaf(-es, es, -e);
        } else {
            float x[I];
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const float z = fmaf(a[i], es, b[i]);
                x[i] = fmaf(-z, z, c[i]);
            }
            float m = x[0];
#pragma unroll
            for (int i = 1; i < I; ++i) m = fmaxf(m, x[i]);
            float sum = 0.0f;
#pragma unroll
            for (int i = 0; i < I; ++i) sum += ex2_approx(x[i] - m);
            u = (m - e) + lg2_approx(sum);
        }
        return u;
    }
    static constexpr double kTermConst = -0.5 * kLog2Pi - kLogSfac;

    template <bool kFirst>
    __device__ __forceinline__ double logdens(float y)
    {
        return kLn2 * (double)logdens2<kFirst>(y) + kTermConst;
    }

    // Closes a 32-observation partial (the product of shifted mixture sums
    // stays below 4^32 = 2^64).
    __device__ __forceinline__ void flush()
    {
        float u = sm - sh;
        if constexpr (I >= 2) u += lg2_approx(prod);
        part += u;
        sh = sm = 0.0f;
        prod = 1.0f;
    }

    // Adds the FP32 partial of up to 256 observations into the FP64 sum.
    __device__ __forceinline__ void flush_fp64()
    {
        acc += (double)part;
        part = 0.0f;
    }

    // log p(y_1:T | theta); call after the last flush.
    __device__ __forceinline__ double finish(int T) const
    {
        return kLn2 * (acc + (double)part) + (double)T * (-0.5 * kLog2Pi - kLogSfac);
    }

    __device__ __forceinline__ void state_out(double* st) const
    {
        st[0] = (double)(kDelta ? v[0] : v[0] - lsy2p) * (2.0 * kLn2);
#pragma unroll
        for (int k = 1; k < K; ++k) st[k] = (double)v[k] * (2.0 * kLn2);
        st[K] = (double)es / kSfac;
    }
};

// ------------------------------------------------------------- FP64 recursion
template <int K, int I>
struct EgarchF64 {
    double mu, lsy;
    double al[K], be[K], ga[K], v0[K];
    double ainv[I], mui[I], lps[I];        // 1/sigma_i, mu_i, log p_i - log sigma_i
    double v[K], eps, acc;

    __device__ __forceinline__ void setup(const double* th, int has_gamma, int eps0_zero)
    {
        EgarchParams<double, K, I> q;
        egarch_transform<double, K, I>(th, has_gamma, q);
        mu = q.mu_y;
        lsy = q.log_sigma_y;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            al[k] = q.alpha[k];
            be[k] = q.beta[k];
            ga[k] = q.gamma[k];
            v0[k] = eps0_zero ? -q.beta[k] * kSqrt2OverPi : 0.0;
        }
#pragma unroll
        for (int i = 0; i < I; ++i) {
            ainv[i] = 1.0 / q.sig[i];
            mui[i] = q.mu[i];
            lps[i] = log(q.p[i]) - log(q.sig[i]);
        }
        eps = 0.0;
        acc = 0.0;
    }

    template <bool kFirst>
    __device__ __forceinline__ void step(double y)
    {
        if constexpr (kFirst) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = v0[k];
        } else {
            const double ae = fabs(eps) - kSqrt2OverPi;
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = al[k] * v[k] + be[k] * ae + ga[k] * eps;
        }
        double vs = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) vs += v[k];
        const double lh = lsy + 0.5 * vs;                 // log h_t
        eps = (y - mu) * exp(-lh);
        double l;
        if constexpr (I == 1) {
            l = -0.5 * eps * eps;
        } else {
            double x[I];
            double m = -INFINITY;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const double z = (eps - mui[i]) * ainv[i];
                x[i] = lps[i] - 0.5 * z * z;
                m = fmax(m, x[i]);
            }
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < I; ++i) s += exp(x[i] - m);
            l = m + log(s);
        }
        acc += l - lh;
    }

    __device__ __forceinline__ void flush() {}

    __device__ __forceinline__ double finish(int T) const
    {
        return acc + (double)T * (-0.5 * kLog2Pi);
    }

    __device__ __forceinline__ void load_state(const double* st)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = st[k];
        eps = st[K];
    }

    template <bool kFirst>
    __device__ __forceinline__ double logdens(double y)
    {
        const double before = acc;
        step<kFirst>(y);
        const double l = acc - before;
        acc = before;
        return l - 0.5 * kLog2Pi;
    }

    __device__ __forceinline__ void state_out(double* st) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k) st[k] = v[k];
        st[K] = eps;
    }
};

// ------------------------------------------------------ observation pipeline
// Double-buffered staging of observation elements into shared memory: chunk c
// lives in buffer c & 1 and is filled by one bulk async copy (plus at most 15
// bytes of tail by plain loads so that no global read passes the end of the
// caller's array).  The buffer is refilled with chunk c + 2 once every thread
// has finished chunk c.
template <typename T, int kChunk>
struct ObsPipe {
    static_assert((kChunk * sizeof(T)) % 16 == 0, "chunk must be a multiple of 16 bytes");
    T* buf;               // [2][kChunk] in shared memory, 16-byte aligned
    uint64_t* bar;        // [2] mbarriers in shared memory
    const T* src;         // global, 16-byte aligned
    int64_t n;            // total elements
    int nchunks;

    __device__ __forceinline__ void issue(int c)
    {
        const int b = c & 1;
        const int64_t off = (int64_t)c * kChunk;
        const int cnt = (int)min((int64_t)kChunk, n - off);
        constexpr int kVec = 16 / (int)sizeof(T);
        const int bulk = cnt & ~(kVec - 1);
        for (int i = bulk; i < cnt; ++i) buf[b * kChunk + i] = src[off + i];
        mbar_arrive_expect_tx(&bar[b], (uint32_t)(bulk * sizeof(T)));
        if (bulk > 0) bulk_copy_g2s(&buf[b * kChunk], src + off, (uint32_t)(bulk * sizeof(T)), &bar[b]);
    }

    // Block-collective start; returns false when there is nothing to stage.
    __device__ __forceinline__ void start()
    {
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0 && nchunks > 0) {
            issue(0);
            if (nchunks > 1) issue(1);
        }
    }

    // Block-collective wait for chunk c.  Returns false (for every thread) if
    // any thread's bounded wait ran out.
    __device__ __forceinline__ bool wait(int c)
    {
        const bool ok = mbar_wait_bounded(&bar[c & 1], (uint32_t)((c >> 1) & 1));
        return !__syncthreads_or(!ok);
    }

    // Block-collective release of chunk c's buffer and refill with chunk c + 2.
    __device__ __forceinline__ void release(int c)
    {
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nchunks) {
            fence_proxy_async_smem();
            issue(c + 2);
        }
    }

    // Block-collective end of use: invalidates the barriers so that the same
    // shared memory can host a new pipeline (persistent kernels).
    __device__ __forceinline__ void finish()
    {
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar[0])) : "memory");
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar[1])) : "memory");
        }
        __syncthreads();
    }

    // After an abandoned wait: give chunks still in flight a bounded chance to
    // land before the block exits.
    __device__ __forceinline__ void drain(int c)
    {
        if (threadIdx.x == 0)
            for (int k = c; k < nchunks && k < c + 2; ++k) mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1));
        __syncthreads();
    }
};

// Observations per chunk of the data-tempering C phase's speculative stop
// search (k_cdata, k_cdata_select).
constexpr int kCdataChunk = 32;

constexpr int kChunkF32 = 1024;   // observations per staged chunk (4 KB)
constexpr int kChunkF64 = 512;    // elements per staged chunk (4 KB)

// Runs the FP32 EGARCH recursion of one particle over T observations staged
// through `pipe`.  Every thread of the block must call it (it contains block
// barriers); `active` selects whose result matters.  Returns false on a
// staging timeout.
template <int K, int I, bool kDelta>
__device__ __forceinline__ bool run_egarch_f32(EgarchF32<K, I, kDelta>& mdl, ObsPipe<float, kChunkF32>& pipe,
                                               int T)
{
    for (int c = 0; c < pipe.nchunks; ++c) {
        if (!pipe.wait(c)) {
            pipe.drain(c);
            return false;
        }
        const float* yb = pipe.buf + (c & 1) * kChunkF32;
        const int cnt = min(kChunkF32, T - c * kChunkF32);
        const int nunits = cnt >> 5;
        for (int u = 0; u < nunits; ++u) {
            const float4* y4 = reinterpret_cast<const float4*>(yb + 32 * u);
            if (c == 0 && u == 0) {
                float4 q = y4[0];
                mdl.template step<true>(q.x);
                mdl.template step<false>(q.y);
                mdl.template step<false>(q.z);
                mdl.template step<false>(q.w);
#pragma unroll
                for (int j = 1; j < 8; ++j) {
                    q = y4[j];
                    mdl.template step<false>(q.x);
                    mdl.template step<false>(q.y);
                    mdl.template step<false>(q.z);
                    mdl.template step<false>(q.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 q = y4[j];
                    mdl.template step<false>(q.x);
                    mdl.template step<false>(q.y);
                    mdl.template step<false>(q.z);
                    mdl.template step<false>(q.w);
                }
            }
            mdl.flush();
            if ((u & 7) == 7) mdl.flush_fp64();
        }
        const int rem = cnt & 31;
        if (rem) {
            for (int r = 0; r < rem; ++r) {
                const int tl = 32 * nunits + r;
                if (c == 0 && tl == 0) mdl.template step<true>(yb[tl]);
                else mdl.template step<false>(yb[tl]);
            }
            mdl.flush();
        }
        pipe.release(c);
    }
    return true;
}

// ------------------------------------------- two particles in packed FP32x2
// Blackwell's paired FP32 instructions (fma/add/mul/sub .f32x2) run the same
// operation on two particles' recursions in one issue slot.  The pair is
// packed from two set-up EgarchF32 models and unpacked back into them, and
// every lane performs exactly the scalar recursion's operations in its order
// (IEEE round-to-nearest per lane), so the results are bitwise those of two
// EgarchF32 runs.  The mixture terms are carried negated where that saves a
// negation: y_i = z_i^2 - c_i = -x_i exactly, max_i x_i = max_i(-y_i),
// x_0 - x_1 = y_1 - y_0.
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b)
{
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

template <int K, int I>
struct EgarchF32Pair {
    float2 nmu;                            // -mu_Y
    float2 al[K], be[K], ga[K], nb[K];
    float2 a[I], b[I], nc[I];              // 1/sigma_i; -mu_i s / sigma_i; -log2(p_i / sigma_i)
    float2 v0[K];
    float2 v[K], es;
    float2 sh, sm, prod;                   // I = 1: sm holds the negated sum
    float part[2];
    double acc[2];

    __device__ __forceinline__ void load(const EgarchF32<K, I>& A, const EgarchF32<K, I>& B)
    {
        nmu = make_float2(-A.mu, -B.mu);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            al[k] = make_float2(A.al[k], B.al[k]);
            be[k] = make_float2(A.be[k], B.be[k]);
            ga[k] = make_float2(A.ga[k], B.ga[k]);
            nb[k] = make_float2(A.nb[k], B.nb[k]);
            v0[k] = make_float2(A.v0[k], B.v0[k]);
            v[k] = make_float2(A.v[k], B.v[k]);
        }
#pragma unroll
        for (int i = 0; i < I; ++i) {
            a[i] = make_float2(A.a[i], B.a[i]);
            b[i] = make_float2(A.b[i], B.b[i]);
            nc[i] = make_float2(-A.c[i], -B.c[i]);
        }
        es = make_float2(A.es, B.es);
        sh = make_float2(A.sh, B.sh);
        sm = I == 1 ? make_float2(-A.sm, -B.sm) : make_float2(A.sm, B.sm);
        prod = make_float2(A.prod, B.prod);
        part[0] = A.part;
        part[1] = B.part;
        acc[0] = A.acc;
        acc[1] = B.acc;
    }

    __device__ __forceinline__ void store(EgarchF32<K, I>& A, EgarchF32<K, I>& B) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            A.v[k] = v[k].x;
            B.v[k] = v[k].y;
        }
        A.es = es.x;
        B.es = es.y;
        A.sh = sh.x;
        B.sh = sh.y;
        A.sm = I == 1 ? -sm.x : sm.x;
        B.sm = I == 1 ? -sm.y : sm.y;
        A.prod = prod.x;
        B.prod = prod.y;
        A.part = part[0];
        B.part = part[1];
        A.acc = acc[0];
        B.acc = acc[1];
    }

    template <bool kFirst>
    __device__ __forceinline__ void step(float y)
    {
        if constexpr (kFirst) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = v0[k];
        } else {
            float2 vp[K];
#pragma unroll
            for (int k = 0; k < K; ++k) vp[k] = f2_fma(al[k], v[k], nb[k]);
            const float2 ae = make_float2(fabsf(es.x), fabsf(es.y));
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = f2_fma(be[k], ae, f2_fma(ga[k], es, vp[k]));
        }
        float2 e = v[0];
#pragma unroll
        for (int k = 1; k < K; ++k) e = f2_add(e, v[k]);
        sh = f2_add(sh, e);
        const float2 ex = make_float2(ex2_approx(-e.x), ex2_approx(-e.y));
        es = f2_mul(f2_add(make_float2(y, y), nmu), ex);
        if constexpr (I == 1) {
            sm = f2_fma(es, es, sm);
        } else if constexpr (I == 2) {
            const float2 z0 = f2_fma(a[0], es, b[0]), z1 = f2_fma(a[1], es, b[1]);
            const float2 y0 = f2_fma(z0, z0, nc[0]), y1 = f2_fma(z1, z1, nc[1]);
            sm = f2_add(sm, make_float2(fmaxf(-y0.x, -y1.x), fmaxf(-y0.y, -y1.y)));
            const float2 dd = f2_sub(y1, y0);
            const float2 r = make_float2(ex2_approx(-fabsf(dd.x)), ex2_approx(-fabsf(dd.y)));
            prod = f2_fma(prod, r, prod);
        } else {
            float2 yv[I];
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const float2 z = f2_fma(a[i], es, b[i]);
                yv[i] = f2_fma(z, z, nc[i]);
            }
            float2 m = make_float2(-yv[0].x, -yv[0].y);
#pragma unroll
            for (int i = 1; i < I; ++i) m = make_float2(fmaxf(m.x, -yv[i].x), fmaxf(m.y, -yv[i].y));
            float2 t = f2_add(yv[0], m);
            float2 ssum = make_float2(ex2_approx(-t.x), ex2_approx(-t.y));
#pragma unroll
            for (int i = 1; i < I; ++i) {
                t = f2_add(yv[i], m);
                ssum = f2_add(ssum, make_float2(ex2_approx(-t.x), ex2_approx(-t.y)));
            }
            sm = f2_add(sm, m);
            prod = f2_mul(prod, ssum);
        }
    }

    // The scalar model's flush, lane by lane.
    __device__ __forceinline__ void flush()
    {
        float u0, u1;
        if constexpr (I == 1) {
            u0 = -(sm.x + sh.x);
            u1 = -(sm.y + sh.y);
        } else {
            u0 = sm.x - sh.x;
            u1 = sm.y - sh.y;
            u0 += lg2_approx(prod.x);
            u1 += lg2_approx(prod.y);
        }
        part[0] += u0;
        part[1] += u1;
        sh = sm = make_float2(0.0f, 0.0f);
        prod = make_float2(1.0f, 1.0f);
    }

    __device__ __forceinline__ void flush_fp64()
    {
        acc[0] += (double)part[0];
        acc[1] += (double)part[1];
        part[0] = part[1] = 0.0f;
    }
};

// Two particles per thread through the packed recursion; A and B hold the
// two models' end states and sums afterwards.
template <int K, int I>
__device__ __forceinline__ bool run_egarch_f32_x2(EgarchF32<K, I>& ma, EgarchF32<K, I>& mb,
                                                  ObsPipe<float, kChunkF32>& pipe, int T)
{
    EgarchF32Pair<K, I> pr;
    pr.load(ma, mb);
    for (int c = 0; c < pipe.nchunks; ++c) {
        if (!pipe.wait(c)) {
            pipe.drain(c);
            pr.store(ma, mb);
            return false;
        }
        const float* yb = pipe.buf + (c & 1) * kChunkF32;
        const int cnt = min(kChunkF32, T - c * kChunkF32);
        const int nunits = cnt >> 5;
        for (int u = 0; u < nunits; ++u) {
            const float4* y4 = reinterpret_cast<const float4*>(yb + 32 * u);
            if (c == 0 && u == 0) {
                float4 q = y4[0];
                pr.template step<true>(q.x);
                pr.template step<false>(q.y);
                pr.template step<false>(q.z);
                pr.template step<false>(q.w);
#pragma unroll
                for (int j = 1; j < 8; ++j) {
                    q = y4[j];
                    pr.template step<false>(q.x);
                    pr.template step<false>(q.y);
                    pr.template step<false>(q.z);
                    pr.template step<false>(q.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 q = y4[j];
                    pr.template step<false>(q.x);
                    pr.template step<false>(q.y);
                    pr.template step<false>(q.z);
                    pr.template step<false>(q.w);
                }
            }
            pr.flush();
            if ((u & 7) == 7) pr.flush_fp64();
        }
        const int rem = cnt & 31;
        if (rem) {
            for (int r = 0; r < rem; ++r) {
                const int tl = 32 * nunits + r;
                if (c == 0 && tl == 0) pr.template step<true>(yb[tl]);
                else pr.template step<false>(yb[tl]);
            }
            pr.flush();
        }
        pipe.release(c);
    }
    pr.store(ma, mb);
    return true;
}

template <int K, int I>
__device__ __forceinline__ bool run_egarch_f64(EgarchF64<K, I>& mdl, ObsPipe<double, kChunkF64>& pipe,
                                               int T)
{
    for (int c = 0; c < pipe.nchunks; ++c) {
        if (!pipe.wait(c)) {
            pipe.drain(c);
            return false;
        }
        const double* yb = pipe.buf + (c & 1) * kChunkF64;
        const int cnt = min(kChunkF64, T - c * kChunkF64);
        int r = 0;
        if (c == 0 && cnt > 0) {
            mdl.template step<true>(yb[0]);
            r = 1;
        }
        for (; r < cnt; ++r) mdl.template step<false>(yb[r]);
        pipe.release(c);
    }
    return true;
}

// Conjugate normal linear regression: y_t = x_t' beta + e_t, e_t ~ N(0, sigma^2)
// with sigma known.  Records are [x_t1 .. x_tp, y_t] (p + 1 doubles).
struct LinregF64 {
    double beta[8];
    int p;
    double inv2s2, c0, isig;
    double acc;

    __device__ __forceinline__ void setup(const double* th, int p_, double sigma)
    {
        p = p_;
        for (int i = 0; i < p; ++i) beta[i] = th[i];
        inv2s2 = 0.5 / (sigma * sigma);
        isig = 1.0 / sigma;
        c0 = -0.5 * kLog2Pi - log(sigma);
        acc = 0.0;
    }

    __device__ __forceinline__ void step(const double* rec)
    {
        double m = 0.0;
        for (int i = 0; i < p; ++i) m += rec[i] * beta[i];
        const double r = rec[p] - m;
        acc += -r * r * inv2s2;
    }

    __device__ __forceinline__ double finish(int T) const { return acc + (double)T * c0; }

    __device__ __forceinline__ double logdens(const double* rec) const
    {
        double m = 0.0;
        for (int i = 0; i < p; ++i) m += rec[i] * beta[i];
        const double r = rec[p] - m;
        return -r * r * inv2s2 + c0;
    }

    // standardized residual (y_t - x_t'beta) / sigma of one record
    __device__ __forceinline__ double shock(const double* rec) const
    {
        double m = 0.0;
        for (int i = 0; i < p; ++i) m += rec[i] * beta[i];
        return (rec[p] - m) * isig;
    }
};

// Records of width W staged in chunks of whole records.
__device__ __forceinline__ bool run_linreg(LinregF64& mdl, ObsPipe<double, kChunkF64>& pipe, int T, int W)
{
    // chunk boundaries fall on record boundaries when kChunkF64 % W == 0; the
    // host restricts W to divisors of kChunkF64 (W in {1, 2, 4, 8}) by padding
    // records with zero columns.
    const int rec_per_chunk = kChunkF64 / W;
    for (int c = 0; c < pipe.nchunks; ++c) {
        if (!pipe.wait(c)) {
            pipe.drain(c);
            return false;
        }
        const double* rb = pipe.buf + (c & 1) * kChunkF64;
        const int nrec = min(rec_per_chunk, T - c * rec_per_chunk);
        for (int r = 0; r < nrec; ++r) mdl.step(rb + r * W);
        pipe.release(c);
    }
    return true;
}

}  // namespace smc
