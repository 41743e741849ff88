// Hot-path kernels: the fused random-walk Metropolis step of the M phase and
// the stand-alone likelihood evaluation, each templated on a model policy.
//
// One thread carries one particle (Section 2.3: "each particle ... in a distinct
// thread").  A block stages the observations once into shared memory with bulk
// async copies and all of its threads run their T-step recursions over the
// same staged values (warp-uniform broadcast reads).
#pragma once

#include "recursion.cuh"

namespace smc {

// Arguments of one M-phase Metropolis iteration (Section 3.3, "Metropolis
// steps"): theta* = theta + L z with L L' = h^2 V, accepted with probability
// min(1, exp{[lp(theta*) + phi l(theta*)] - [lp(theta) + phi l(theta)]}).
struct MutateArgs {
    ModelDev m;
    const void* obs;        // observation records (float for FP32 EGARCH, double otherwise)
    int T;                  // records used (t_l in data tempering, T in power tempering)
    int W;                  // doubles per record (LINREG), 1 otherwise
    double* theta;          // [d][P]
    double* ll;             // [P]
    double* lp;             // [P]
    double* state;          // [ns][P] (nullable)
    double* thp;            // [d][P] proposal scratch
    int P;
    int ns;
    const double* L;        // [d][d] lower Cholesky factor of h^2 V, row-major
    double phi;
    uint64_t seed, cycle, iter;
    unsigned long long* acc_count;   // += accepted proposals
    int* err;
};

struct LoglikArgs {
    ModelDev m;
    const void* obs;
    int T, W;
    const double* theta;    // [d][P]
    double* ll;             // [P]
    double* lp;             // [P] (nullable)
    double* state;          // [ns][P] (nullable)
    int P, ns;
    int* err;
};

constexpr int kMutThreads = 128;

template <int K, int I>
struct PolicyEgarchF32 {
    using Real = float;
    using Obs = float;
    static constexpr int kChunk = kChunkF32;
    using Model = EgarchF32<K, I>;
    static constexpr int kNs = K + 1;
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.gamma, m.eps0_zero);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int) { return run_egarch_f32(mdl, pipe, T); }
    __device__ static void state_out(const Model& mdl, double* st) { mdl.state_out(st); }
};

template <int K, int I>
struct PolicyEgarchF64 {
    using Real = double;
    using Obs = double;
    static constexpr int kChunk = kChunkF64;
    using Model = EgarchF64<K, I>;
    static constexpr int kNs = K + 1;
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.gamma, m.eps0_zero);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int) { return run_egarch_f64(mdl, pipe, T); }
    __device__ static void state_out(const Model& mdl, double* st) { mdl.state_out(st); }
};

struct PolicyLinreg {
    using Real = double;
    using Obs = double;
    static constexpr int kChunk = kChunkF64;
    using Model = LinregF64;
    static constexpr int kNs = 0;
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.p, m.sigma);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int W) { return run_linreg(mdl, pipe, T, W); }
    __device__ static void state_out(const Model&, double*) {}
};

__device__ __forceinline__ double tempered_target(double lp, double ll, double phi)
{
    if (lp == -INFINITY) return -INFINITY;
    return phi > 0.0 ? lp + phi * ll : lp;
}

template <class Pol>
__global__ void __launch_bounds__(kMutThreads) k_mutate(MutateArgs a)
{
    using Real = typename Pol::Real;
    using Obs = typename Pol::Obs;
    __shared__ __align__(16) Obs obuf[2 * Pol::kChunk];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ Real Ls[kMaxD * kMaxD];
    __shared__ unsigned int acc_s;

    const int d = a.m.d;
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) Ls[i] = (Real)a.L[i];
    if (threadIdx.x == 0) acc_s = 0;

    const int64_t nelem = (int64_t)a.T * a.W;
    ObsPipe<Obs, Pol::kChunk> pipe{obuf, bars, (const Obs*)a.obs, nelem,
                                   (int)((nelem + Pol::kChunk - 1) / Pol::kChunk)};
    pipe.start();   // contains a block barrier: Ls and acc_s are visible below

    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < a.P;
    const int pp = active ? p : a.P - 1;
    const size_t P = (size_t)a.P;

    // Proposal theta* = theta + L z (Section 3.3), written to the scratch rows.
    double thn[kMaxD];
    {
        Real z[kMaxD];
        proposal_normals<Real>(a.seed, (uint64_t)pp, a.iter, a.cycle, d, z);
        for (int i = 0; i < d; ++i) {
            Real s = 0;
            for (int k = 0; k <= i; ++k) s += Ls[i * d + k] * z[k];
            thn[i] = a.theta[i * P + pp] + (double)s;
            if (active) a.thp[i * P + p] = thn[i];
        }
    }
    const double lp_new = log_prior(a.m, thn);
    typename Pol::Model mdl;
    {
        Real full[kMaxD];
        full_theta<Real>(a.m, thn, full);
        Pol::setup(mdl, a.m, full);
    }
    const bool ok = Pol::run(mdl, pipe, a.T, a.W);
    double ll_new = ok ? mdl.finish(a.T) : -INFINITY;
    if (isnan(ll_new)) ll_new = -INFINITY;
    if (!ok && threadIdx.x == 0) raise_error(a.err, kErrTimeout);

    bool acc = false;
    if (active) {
        const double log_alpha = tempered_target(lp_new, ll_new, a.phi) -
                                 tempered_target(a.lp[p], a.ll[p], a.phi);
        const double log_u = log_uniform_mh(a.seed, (uint64_t)p, a.iter, a.cycle);
        acc = log_u < log_alpha;
        if (acc) {
            for (int i = 0; i < d; ++i) a.theta[i * P + p] = a.thp[i * P + p];
            a.ll[p] = ll_new;
            a.lp[p] = lp_new;
            if (a.state) {
                double st[kMaxState];
                Pol::state_out(mdl, st);
                for (int k = 0; k < Pol::kNs; ++k) a.state[k * P + p] = st[k];
            }
        }
    }
    const unsigned int nacc = __popc(__ballot_sync(0xffffffffu, acc));
    if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&acc_s, nacc);
    __syncthreads();
    if (threadIdx.x == 0 && acc_s) atomicAdd(a.acc_count, (unsigned long long)acc_s);
}

template <class Pol>
__global__ void __launch_bounds__(kMutThreads) k_loglik(LoglikArgs a)
{
    using Real = typename Pol::Real;
    using Obs = typename Pol::Obs;
    __shared__ __align__(16) Obs obuf[2 * Pol::kChunk];
    __shared__ __align__(8) uint64_t bars[2];

    const int64_t nelem = (int64_t)a.T * a.W;
    ObsPipe<Obs, Pol::kChunk> pipe{obuf, bars, (const Obs*)a.obs, nelem,
                                   (int)((nelem + Pol::kChunk - 1) / Pol::kChunk)};
    pipe.start();

    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < a.P;
    const int pp = active ? p : a.P - 1;
    const size_t P = (size_t)a.P;
    const int d = a.m.d;

    double th[kMaxD];
    for (int i = 0; i < d; ++i) th[i] = a.theta[i * P + pp];
    typename Pol::Model mdl;
    {
        Real full[kMaxD];
        full_theta<Real>(a.m, th, full);
        Pol::setup(mdl, a.m, full);
    }
    const bool ok = Pol::run(mdl, pipe, a.T, a.W);
    double ll = ok ? mdl.finish(a.T) : -INFINITY;
    if (isnan(ll)) ll = -INFINITY;
    if (!ok && threadIdx.x == 0) raise_error(a.err, kErrTimeout);
    if (active) {
        a.ll[p] = ll;
        if (a.lp) a.lp[p] = log_prior(a.m, th);
        if (a.state) {
            double st[kMaxState];
            Pol::state_out(mdl, st);
            for (int k = 0; k < Pol::kNs; ++k) a.state[k * P + p] = st[k];
        }
    }
}

// Host-side launchers (defined in the instantiation units).
cudaError_t launch_mutate(const MutateArgs& a, int precision, cudaStream_t s);
cudaError_t launch_loglik(const LoglikArgs& a, int precision, cudaStream_t s);

}  // namespace smc
