// Gradient kernel (log likelihood and its theta-gradient per particle) and the
// fused MALA mutation kernel, templated on a gradient policy.
#pragma once

#include "adjoint.cuh"
#include "kernels.cuh"

namespace smc {

constexpr int kMalaThreads = 128;
// Launch width of the gradient kernels: each thread holds a shared-memory slab
// for one segment's recomputed states (mala_seg x (K + 2) values), so narrower blocks
// pack more resident blocks per SM and leave a smaller last wave.
constexpr int kMalaLaunch = 64;

struct GradArgs {
    ModelDev m;
    const void* obs;
    int T, W;
    const double* theta;   // [d][P]
    int P;
    double* ll;            // [P]
    double* grad;          // [d][P] d log p(y|theta) / d theta (free parameters)
    double* state;         // [K+1][P] (nullable)
    void* ckpt;            // segment checkpoints (gradient policy's layout)
};

// One MALA iteration: theta* = theta + (1/2) L L' g + L z with g the gradient
// of the tempered log target lp + phi l at theta (from the stored likelihood
// gradient), accepted with the Metropolis-Hastings ratio including
// q(theta | theta*) / q(theta* | theta).
struct MalaArgs {
    ModelDev m;
    const void* obs;
    int T, W;
    double* theta;         // [d][P]
    double* ll;            // [P]
    double* lp;            // [P]
    double* state;         // [ns][P] (nullable)
    double* grad;          // [d][P] likelihood gradient at the current particles
    void* ckpt;            // segment checkpoints of the proposal's recursion
    int P, ns;
    const double* L;       // [d][d]
    double phi;
    uint64_t seed, cycle, iter;
    unsigned long long* acc_count;
    int* pending;
    int* err;
};

// Observations per checkpoint segment of the EGARCH adjoint (the reverse
// sweep's shared-memory slab holds one segment per thread); the checkpoint
// buffers are sized from the same value.  (16 in FP32 as well, for more
// resident blocks, was measured and not kept: 5.81 against 5.90 ms per launch
// at K=2, I=2, T=5000, 262,144 particles, for twice the checkpoint memory.)
template <typename Real>
constexpr int mala_seg() { return sizeof(Real) == 4 ? 32 : 16; }

template <typename Real, int K, int I>
struct GradEgarch {
    using RealT = Real;
    static constexpr int kSeg = mala_seg<Real>();
    static constexpr int kNs = K + 1;
    static size_t smem_bytes(int threads) { return (size_t)kSeg * (K + 2) * threads * sizeof(Real); }
    static size_t ckpt_bytes(int T, int P)
    {
        const int nseg = (T + kSeg - 1) / kSeg;
        return (size_t)(nseg > 1 ? nseg - 1 : 1) * (K + 1) * (size_t)P * sizeof(Real);
    }
    __device__ static double eval(const ModelDev& m, const double* th, const void* obs, int T, int,
                                  void* ckpt, size_t P, int p, Real* buf, int stride, double* g,
                                  double* st)
    {
        Real full[kMaxD];
        full_theta<Real>(m, th, full);
        EgarchNat<Real, K, I> mdl;
        mdl.setup(full, m.gamma, m.eps0_zero);
        const Real* y = (const Real*)obs;
        double ll;
        if constexpr (sizeof(Real) == 4) {
            ll = adj_forward_fast<K, I, kSeg>(full, m.gamma, m.eps0_zero, y, T, (Real*)ckpt, P, p);
            // end state: recompute the last segment's tail from its checkpoint
            const int nseg = (T + kSeg - 1) / kSeg;
            if (nseg > 1) {
                const Real* c = (const Real*)ckpt + (size_t)(nseg - 2) * (K + 1) * P + p;
#pragma unroll
                for (int k = 0; k < K; ++k) mdl.v[k] = c[k * P];
                mdl.eps = c[K * P];
            }
            for (int t = (nseg - 1) * kSeg; t < T; ++t) {
                Real inv;
                if (t == 0) mdl.template step_state<true>(y[0], inv);
                else mdl.template step_state<false>(y[t], inv);
            }
        } else {
            ll = adj_forward<Real, K, I, kSeg>(mdl, y, T, (Real*)ckpt, P, p, true);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) st[k] = (double)mdl.v[k];
        st[K] = (double)mdl.eps;
        double gn[EgarchNat<Real, K, I>::kNp];
        adj_reverse<Real, K, I, kSeg>(mdl, y, T, (const Real*)ckpt, P, p, buf, stride, gn);
        double gfull[kMaxD];
        natural_to_theta<Real, K, I>(mdl, gn, full, m.gamma, gfull);
        if (m.has_free)
            for (int k = 0; k < m.d; ++k) g[k] = gfull[m.free_idx[k]];
        else
            for (int k = 0; k < m.d; ++k) g[k] = gfull[k];
        if (!(ll > -INFINITY) || isnan(ll)) ll = -INFINITY;
        return ll;
    }
};

// Conjugate regression: l = sum_t [-(y_t - x_t'b)^2 / 2 sigma^2] + T c,
// dl/db = sum_t (y_t - x_t'b) x_t / sigma^2.
struct GradLinreg {
    using RealT = double;
    static constexpr int kNs = 0;
    static size_t smem_bytes(int) { return 0; }
    static size_t ckpt_bytes(int, int) { return 8; }
    __device__ static double eval(const ModelDev& m, const double* th, const void* obs, int T, int W,
                                  void*, size_t, int, double*, int, double* g, double*)
    {
        const double* rec = (const double*)obs;
        const double is2 = 1.0 / (m.sigma * m.sigma);
        double acc = 0.0;
        double gg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < T; ++t) {
            const double* r = rec + (size_t)t * W;
            double mu = 0.0;
            for (int i = 0; i < m.p; ++i) mu += r[i] * th[i];
            const double e = r[m.p] - mu;
            acc -= 0.5 * e * e * is2;
            for (int i = 0; i < m.p; ++i) gg[i] += e * r[i] * is2;
        }
        for (int i = 0; i < m.p; ++i) g[i] = gg[i];
        return acc + (double)T * (-0.5 * kLog2Pi - log(m.sigma));
    }
};

__device__ __forceinline__ void log_prior_grad(const ModelDev& m, const double* th, double* g)
{
    for (int k = 0; k < m.d; ++k) {
        const double s = m.prior_isd[k];
        g[k] = -(th[k] - m.prior_mean[k]) * s * s;
    }
}

template <class GP>
__global__ void __launch_bounds__(kMalaThreads) k_loglik_grad(GradArgs a)
{
    using Real = typename GP::RealT;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const size_t P = (size_t)a.P;
    Real* buf = reinterpret_cast<Real*>(sm_raw) + threadIdx.x;
    double th[kMaxD], g[kMaxD], st[kMaxState];
    for (int i = 0; i < a.m.d; ++i) th[i] = a.theta[i * P + p];
    const double ll = GP::eval(a.m, th, a.obs, a.T, a.W, a.ckpt, P, p, buf, blockDim.x, g, st);
    a.ll[p] = ll;
    for (int i = 0; i < a.m.d; ++i) a.grad[i * P + p] = g[i];
    if (a.state)
        for (int k = 0; k < GP::kNs; ++k) a.state[k * P + p] = st[k];
}

// One particle's MALA iteration (the body of k_mutate_mala and of the batched
// persistent kernel): proposal with the drift (1/2) L L' g, log likelihood and
// gradient of the proposal, the Metropolis-Hastings ratio with the reverse
// proposal density, and on acceptance the write-back of theta, gradient, log
// likelihood, log prior and state.  Ls: L in the working precision (shared
// memory); buf/stride: this thread's segment slab.  Returns the decision.
template <class GP>
__device__ __forceinline__ bool mala_particle(const MalaArgs& a, uint64_t iter, int p,
                                              const typename GP::RealT* Ls, typename GP::RealT* buf, int stride)
{
    using Real = typename GP::RealT;
    const int d = a.m.d;
    const size_t P = (size_t)a.P;
    double th[kMaxD], g[kMaxD], prop[kMaxD];
    Real z[kMaxD], w[kMaxD];
    for (int i = 0; i < d; ++i) th[i] = a.theta[i * P + p];
    // gradient of the tempered log target at theta
    log_prior_grad(a.m, th, g);
    for (int i = 0; i < d; ++i) g[i] += a.phi * a.grad[i * P + p];
    // drift (1/2) L (L' g) and proposal
    for (int k = 0; k < d; ++k) {
        Real s = 0;
        for (int i = k; i < d; ++i) s += Ls[i * d + k] * (Real)g[i];
        w[k] = s;
    }
    proposal_normals<Real>(a.seed, (uint64_t)p, iter, a.cycle, d, z);
    Real zz = 0;
    for (int i = 0; i < d; ++i) {
        Real s1 = 0, s2 = 0;
        for (int k = 0; k <= i; ++k) {
            s1 += Ls[i * d + k] * w[k];
            s2 += Ls[i * d + k] * z[k];
        }
        prop[i] = th[i] + (double)(Real(0.5) * s1 + s2);
        zz += z[i] * z[i];
    }
    const double lp_new = log_prior(a.m, prop);
    double gl[kMaxD], st[kMaxState];
    const double ll_new = GP::eval(a.m, prop, a.obs, a.T, a.W, a.ckpt, P, p, buf, stride, gl, st);
    double log_alpha = -INFINITY;
    if (lp_new > -INFINITY && ll_new > -INFINITY) {
        double g2[kMaxD];
        log_prior_grad(a.m, prop, g2);
        for (int i = 0; i < d; ++i) g2[i] += a.phi * gl[i];
        for (int k = 0; k < d; ++k) {
            Real s = 0;
            for (int i = k; i < d; ++i) s += Ls[i * d + k] * (Real)g2[i];
            w[k] = s;
        }
        // u = L^-1 (theta - theta* - (1/2) L L' g*), zero pivots contribute nothing
        double uu = 0.0;
        Real u[kMaxD];
        for (int i = 0; i < d; ++i) {
            Real s1 = 0;
            for (int k = 0; k <= i; ++k) s1 += Ls[i * d + k] * w[k];
            Real r = (Real)(th[i] - prop[i]) - Real(0.5) * s1;
            for (int k = 0; k < i; ++k) r -= Ls[i * d + k] * u[k];
            u[i] = Ls[i * d + i] > Real(0) ? r / Ls[i * d + i] : Real(0);
            uu += (double)u[i] * (double)u[i];
        }
        log_alpha = tempered_target(lp_new, ll_new, a.phi) - tempered_target(a.lp[p], a.ll[p], a.phi) -
                    0.5 * uu + 0.5 * (double)zz;
    }
    const bool acc = mh_accept(a.seed, (uint64_t)p, iter, a.cycle, log_alpha);
    if (acc) {
        for (int i = 0; i < d; ++i) {
            a.theta[i * P + p] = prop[i];
            a.grad[i * P + p] = gl[i];
        }
        a.ll[p] = ll_new;
        a.lp[p] = lp_new;
        if (a.state)
            for (int k = 0; k < GP::kNs; ++k) a.state[k * P + p] = st[k];
    }
    return acc;
}

template <class GP>
__global__ void __launch_bounds__(kMalaThreads) k_mutate_mala(MalaArgs a)
{
    using Real = typename GP::RealT;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ Real Ls[kMaxD * kMaxD];
    __shared__ unsigned int acc_s;
    const int d = a.m.d;
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) Ls[i] = (Real)a.L[i];
    if (threadIdx.x == 0) acc_s = 0;
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool acc = false;
    if (p < a.P) acc = mala_particle<GP>(a, a.iter, p, Ls, reinterpret_cast<Real*>(sm_raw) + threadIdx.x,
                                         blockDim.x);
    const unsigned int nacc = __popc(__ballot_sync(0xffffffffu, acc));
    if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&acc_s, nacc);
    __syncthreads();
    if (threadIdx.x == 0 && acc_s) atomicAdd(a.acc_count, (unsigned long long)acc_s);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.pending) *a.pending = 1;
}

template <class GP>
cudaError_t launch_grad_t(const GradArgs& a, cudaStream_t s)
{
    const size_t sm = GP::smem_bytes(kMalaLaunch);
    static bool attr = false;
    if (!attr && sm > 0) {   // static + dynamic shared memory may pass the 48 KB default
        cudaFuncSetAttribute(k_loglik_grad<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    k_loglik_grad<GP><<<(a.P + kMalaLaunch - 1) / kMalaLaunch, kMalaLaunch, sm, s>>>(a);
    return cudaGetLastError();
}

template <class GP>
cudaError_t launch_mala_t(const MalaArgs& a, cudaStream_t s)
{
    const size_t sm = GP::smem_bytes(kMalaLaunch);
    static bool attr = false;
    if (!attr && sm > 0) {   // static + dynamic shared memory may pass the 48 KB default
        cudaFuncSetAttribute(k_mutate_mala<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    k_mutate_mala<GP><<<(a.P + kMalaLaunch - 1) / kMalaLaunch, kMalaLaunch, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename Real, int K>
cudaError_t launch_grad_k(const GradArgs& a, cudaStream_t s)
{
    switch (a.m.I) {
    case 1: return launch_grad_t<GradEgarch<Real, K, 1>>(a, s);
    case 2: return launch_grad_t<GradEgarch<Real, K, 2>>(a, s);
    case 3: return launch_grad_t<GradEgarch<Real, K, 3>>(a, s);
    case 4: return launch_grad_t<GradEgarch<Real, K, 4>>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename Real, int K>
cudaError_t launch_mala_k(const MalaArgs& a, cudaStream_t s)
{
    switch (a.m.I) {
    case 1: return launch_mala_t<GradEgarch<Real, K, 1>>(a, s);
    case 2: return launch_mala_t<GradEgarch<Real, K, 2>>(a, s);
    case 3: return launch_mala_t<GradEgarch<Real, K, 3>>(a, s);
    case 4: return launch_mala_t<GradEgarch<Real, K, 4>>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_loglik_grad(const GradArgs& a, int precision, cudaStream_t s);
cudaError_t launch_mala(const MalaArgs& a, int precision, cudaStream_t s);
inline size_t mala_ckpt_bytes(const ModelDev& m, int precision, int T, int P)
{
    if (m.kind == 1) return GradLinreg::ckpt_bytes(T, P);
    const size_t real = precision == 1 ? 4 : 8;
    const int seg = precision == 1 ? mala_seg<float>() : mala_seg<double>();
    const int nseg = (T + seg - 1) / seg;
    return (size_t)(nseg > 1 ? nseg - 1 : 1) * (m.K + 1) * (size_t)P * real;
}

}  // namespace smc
