// Hot-path kernels: the fused random-walk Metropolis step of the M phase and
// the stand-alone likelihood evaluation, each templated on a model policy.
//
// One thread carries one particle (Section 2.3: "each particle ... in a distinct
// thread").  A block stages the observations once into shared memory with bulk
// async copies and all of its threads run their T-step recursions over the
// same staged values (warp-uniform broadcast reads).
#pragma once

#include "recursion.cuh"
#include "covtile.cuh"

namespace smc {

// Arguments of one M-phase Metropolis iteration (Section 3.3, "Metropolis
// steps"): theta* = theta + L z with L L' = h^2 V, accepted with probability
// min(1, exp{[lp(theta*) + phi l(theta*)] - [lp(theta) + phi l(theta)]}).
// With qmean set, the independent Gaussian sampler of the same passage:
// theta* = qmean + L z (L L' = V), and the ratio also carries
// log q(theta) - log q(theta*) for q = N(qmean, L L'); log q(theta) comes
// precomputed per particle (launch_indep_logq), log q(theta*) = -|z|^2 / 2.
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
    const double* qmean;    // [d] independent-sampler mean (nullptr: random walk)
    // Covariance of the next iteration (nullable): per 32-particle tile, FP32
    // sums of theta_i - covshift_i and of their products over the tile's
    // particles after this iteration's decision, entry-major
    // [kD + kD(kD+1)/2][ntiles] with kD the policy's parameter bound.
    float* covtile;
    const float* covshift;  // [d] the tiles' shift (the pooled mean rounded to FP32)
    int ntiles;
    const double* lq;       // [P] independent sampler: log q(theta) of the current particles
    double phi;
    uint64_t seed, cycle, iter;
    unsigned long long* acc_count;   // += accepted proposals
    int* pending;                    // set to 1 (nullable): an acceptance count awaits its h update
    int* err;
    // Host-side launch choice: nonzero launches the kernel as a programmatic
    // dependent of the preceding kernel (the covariance step lets it launch
    // once only its final block remains).
    int dependent = 0;
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
// Largest mutation block (threads, a multiple of 32): any multiple of 32 up to
// this is a valid launch shape, so that P particles can be spread as evenly
// as the warp granularity allows over the SMs.  The launch bounds also steer
// the register allocation, and with it the speed (measured on the FP32
// EGARCH(2,2) kernels, 65,536 particles in 224-thread blocks): one particle
// per thread is fastest compiled for 256-thread blocks (48 registers,
// 0.282 ms per launch against 0.292 ms with 56 registers under a 224 or
// 128 bound, 0.288 ms at a 64-register cap), two per thread for 224 (111
// registers, 0.297 ms; 80 registers under a 256 bound: 0.307 ms).
constexpr int kMutMaxThreads = 224;
constexpr int kMutBoundX1 = 256;

// Probability integral transform draw (Section 4.1): the standardized shock
// of Y_s ~ p(Y_s | y_1:s-1, theta), location + scale * e, so that
// I[Y_s <= y_s] = I[e <= e_s].  The Philox block at counter
// (particle, s, 0, kTagPit << 32) gives a uniform that picks mixture component
// i when it falls below p_1 + .. + p_i (first such i), and two uniforms for a
// Box-Muller normal z; e = mu_i + sigma_i z.
template <typename Real, int I>
struct PitMixture {
    double cum[I];
    Real mu[I], sig[I];

    __device__ __forceinline__ double shock(uint64_t seed, uint64_t p, int s) const
    {
        const U64x4 r = philox4x64_10(p, (uint64_t)s, 0, (uint64_t)kTagPit << 32, seed, 0);
        const double uc = uniform53(r.v0);
        Real z;
        if constexpr (sizeof(Real) == 8) {
            z = sqrt(-2.0 * log(uniform53(r.v1))) * cospi(2.0 * uniform53(r.v2));
        } else {
            const float ua = ((float)(uint32_t)(r.v1 >> 40) + 0.5f) * 0x1.0p-24f;
            const float ub = ((float)(uint32_t)(r.v2 >> 40) + 0.5f) * 0x1.0p-24f;
            z = sqrtf(-2.0f * logf(ua)) * cospif(2.0f * ub);
        }
        Real m = mu[I - 1], sg = sig[I - 1];
        bool found = false;
#pragma unroll
        for (int i = 0; i < I; ++i) {
            if (!found && uc < cum[i]) {
                m = mu[i];
                sg = sig[i];
                found = true;
            }
        }
        return (double)(m + sg * z);
    }
};

template <typename Real, int K, int I>
__device__ __forceinline__ void pit_setup_egarch(const ModelDev& m, const double* th, PitMixture<Real, I>& pm)
{
    Real full[kMaxD];
    full_theta<Real>(m, th, full);
    EgarchParams<Real, K, I> q;
    egarch_transform<Real, K, I>(full, m.gamma, q);
    double c = 0.0;
#pragma unroll
    for (int i = 0; i < I; ++i) {
        c += (double)q.p[i];
        pm.cum[i] = c;
        pm.mu[i] = q.mu[i];
        pm.sig[i] = q.sig[i];
    }
}

template <int K, int I, bool kDelta>
struct PolicyEgarchF32T {
    using Real = float;
    using Obs = float;
    static constexpr int kChunk = kChunkF32;
    using Model = EgarchF32<K, I, kDelta>;
    static constexpr int kNs = K + 1;
    static constexpr int kMaxFree = I == 1 ? 2 + 3 * K : 2 + 3 * K + 3 * I;   // Table 1
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.gamma, m.eps0_zero);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int) { return run_egarch_f32(mdl, pipe, T); }
    __device__ static void state_out(const Model& mdl, double* st) { mdl.state_out(st); }
    __device__ static void load_state(Model& mdl, const double* st) { mdl.load_state(st); }
    __device__ static double logdens(Model& mdl, const Obs* obs, int s, int)
    {
        const Obs y = obs[s - 1];
        return s == 1 ? mdl.template logdens<true>(y) : mdl.template logdens<false>(y);
    }
    // The data-tempering C phase can keep its per-observation terms in log2
    // units (l_s = ln2 u_s + kTermConst) and sum them on the FP32 pipe.
    static constexpr bool kLog2Terms = true;
    static constexpr double kTermConst = Model::kTermConst;
    __device__ static float logdens2(Model& mdl, const Obs* obs, int s, int)
    {
        const Obs y = obs[s - 1];
        return s == 1 ? mdl.template logdens2<true>(y) : mdl.template logdens2<false>(y);
    }
    using Pit = PitMixture<float, I>;
    __device__ static void pit_setup(const ModelDev& m, const double* th, Pit& pm) { pit_setup_egarch<float, K, I>(m, th, pm); }
    // observed standardized shock after logdens of observation s
    __device__ static double obs_shock(const Model& mdl, const Obs*, int, int) { return (double)mdl.es * (1.0 / kSfac); }
};

// The FP32 recursion of the M phase (alpha v as one FMA) and, for the kernels
// that see raw prior draws (the stand-alone likelihood and the data-tempering
// C phase), the form that carries 1 - alpha (EgarchF32's kDelta).
template <int K, int I>
struct PolicyEgarchF32 : PolicyEgarchF32T<K, I, false> {};
template <int K, int I>
struct PolicyEgarchF32Delta : PolicyEgarchF32T<K, I, true> {};

template <int K, int I>
struct PolicyEgarchF64 {
    using Real = double;
    using Obs = double;
    static constexpr int kChunk = kChunkF64;
    using Model = EgarchF64<K, I>;
    static constexpr int kNs = K + 1;
    static constexpr int kMaxFree = I == 1 ? 2 + 3 * K : 2 + 3 * K + 3 * I;
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.gamma, m.eps0_zero);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int) { return run_egarch_f64(mdl, pipe, T); }
    __device__ static void state_out(const Model& mdl, double* st) { mdl.state_out(st); }
    __device__ static void load_state(Model& mdl, const double* st) { mdl.load_state(st); }
    __device__ static double logdens(Model& mdl, const Obs* obs, int s, int)
    {
        const Obs y = obs[s - 1];
        return s == 1 ? mdl.template logdens<true>(y) : mdl.template logdens<false>(y);
    }
    static constexpr bool kLog2Terms = false;
    static constexpr double kTermConst = 0.0;
    __device__ static float logdens2(Model&, const Obs*, int, int) { return 0.0f; }
    using Pit = PitMixture<double, I>;
    __device__ static void pit_setup(const ModelDev& m, const double* th, Pit& pm) { pit_setup_egarch<double, K, I>(m, th, pm); }
    __device__ static double obs_shock(const Model& mdl, const Obs*, int, int) { return mdl.eps; }
};

struct PolicyLinreg {
    using Real = double;
    using Obs = double;
    static constexpr int kChunk = kChunkF64;
    using Model = LinregF64;
    static constexpr int kNs = 0;
    static constexpr int kMaxFree = 8;
    __device__ static void setup(Model& mdl, const ModelDev& m, const Real* full)
    {
        mdl.setup(full, m.p, m.sigma);
    }
    __device__ static bool run(Model& mdl, ObsPipe<Obs, kChunk>& pipe, int T, int W) { return run_linreg(mdl, pipe, T, W); }
    __device__ static void state_out(const Model&, double*) {}
    __device__ static void load_state(Model&, const double*) {}
    __device__ static double logdens(Model& mdl, const Obs* obs, int s, int W)
    {
        return mdl.logdens(obs + (size_t)(s - 1) * W);
    }
    static constexpr bool kLog2Terms = false;
    static constexpr double kTermConst = 0.0;
    __device__ static float logdens2(Model&, const Obs*, int, int) { return 0.0f; }
    using Pit = PitMixture<double, 1>;
    __device__ static void pit_setup(const ModelDev&, const double*, Pit& pm)
    {
        pm.cum[0] = 1.0;
        pm.mu[0] = 0.0;
        pm.sig[0] = 1.0;
    }
    __device__ static double obs_shock(const Model& mdl, const Obs* obs, int s, int W)
    {
        return mdl.shock(obs + (size_t)(s - 1) * W);
    }
};

__device__ __forceinline__ double tempered_target(double lp, double ll, double phi)
{
    if (lp == -INFINITY) return -INFINITY;
    return phi > 0.0 ? lp + phi * ll : lp;
}


// Shared memory of one mutation tile.
template <class Pol>
struct MutateSmem {
    __align__(16) typename Pol::Obs obuf[2 * Pol::kChunk];
    __align__(8) uint64_t bars[2];
    typename Pol::Real Ls[kMaxD * kMaxD];
    unsigned int acc_s;
};

template <int kD>
__device__ __forceinline__ void cov_tile_sums(const MutateArgs& a, int p, bool active)
{
    cov_tile_sums<kD>(a.theta, (size_t)a.P, a.m.d, a.covshift, a.covtile, a.ntiles, p, active);
}

// One block's tile of particles p0 + threadIdx.x: proposal, likelihood
// recursion over the staged observations, Metropolis-Hastings decision.
// Every thread of the block must call it (block barriers inside).  kIndep
// selects the independent sampler (a.qmean, a.lq set) at compile time, so the
// random-walk instantiation carries none of its code.
template <class Pol, bool kIndep = false>
__device__ __forceinline__ void mutate_tile(const MutateArgs& a, uint64_t iter, int p0, MutateSmem<Pol>& sm)
{
    using Real = typename Pol::Real;
    using Obs = typename Pol::Obs;
    const int d = a.m.d;
    pdl_wait();   // under a dependent launch: nothing the covariance step writes is read before this
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) sm.Ls[i] = (Real)a.L[i];
    if (threadIdx.x == 0) sm.acc_s = 0;

    const int64_t nelem = (int64_t)a.T * a.W;
    ObsPipe<Obs, Pol::kChunk> pipe{sm.obuf, sm.bars, (const Obs*)a.obs, nelem,
                                   (int)((nelem + Pol::kChunk - 1) / Pol::kChunk)};
    pipe.start();   // contains a block barrier: Ls and acc_s are visible below

    const int p = p0 + (int)threadIdx.x;
    const bool active = p < a.P;
    const int pp = active ? p : a.P - 1;
    const size_t P = (size_t)a.P;

    // Proposal theta* = theta + L z, or qmean + L z for the independent
    // sampler (Section 3.3), written to the scratch rows.
    double thn[kMaxD];
    double zz = 0.0;
    Real thr[kMaxD];   // the proposal in the working precision
    {
        Real z[kMaxD];
        proposal_normals<Real>(a.seed, (uint64_t)pp, iter, a.cycle, d, z);
        for (int i = 0; i < d; ++i) {
            Real s = 0;
            for (int k = 0; k <= i; ++k) s += sm.Ls[i * d + k] * z[k];
            if constexpr (kIndep) {
                thn[i] = a.qmean[i] + (double)s;
                zz += (double)z[i] * (double)z[i];
            } else {
                thn[i] = a.theta[i * P + pp] + (double)s;
            }
            thr[i] = (Real)thn[i];
            if (active) a.thp[i * P + p] = thn[i];
        }
    }
    double lp_new;
    typename Pol::Model mdl;
    {
        Real full[kMaxD];
        if constexpr (sizeof(Real) == 4) {
            lp_new = log_prior_f(a.m, thn, thr);
            full_theta_f(a.m, thr, full);
        } else {
            lp_new = log_prior(a.m, thn);
            full_theta<Real>(a.m, thn, full);
        }
        Pol::setup(mdl, a.m, full);
    }
    const bool ok = Pol::run(mdl, pipe, a.T, a.W);
    pdl_trigger();   // the covariance step that follows may launch once every block is here
    double ll_new = ok ? mdl.finish(a.T) : -INFINITY;
    if (isnan(ll_new)) ll_new = -INFINITY;
    if (!ok && threadIdx.x == 0) raise_error(a.err, kErrTimeout);

    bool acc = false;
    if (active) {
        double log_alpha = tempered_target(lp_new, ll_new, a.phi) -
                           tempered_target(a.lp[p], a.ll[p], a.phi);
        if constexpr (kIndep) log_alpha += a.lq[p] + 0.5 * zz;
        acc = mh_accept(a.seed, (uint64_t)p, iter, a.cycle, log_alpha);
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
    if (a.covtile) cov_tile_sums<Pol::kMaxFree>(a, p, active);
    if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&sm.acc_s, nacc);
    __syncthreads();
    if (threadIdx.x == 0 && sm.acc_s) atomicAdd(a.acc_count, (unsigned long long)sm.acc_s);
    if (p0 == 0 && threadIdx.x == 0 && a.pending) *a.pending = 1;
    pipe.finish();
}

template <class Pol, bool kIndep = false>
__global__ void __launch_bounds__(kMutBoundX1) k_mutate(MutateArgs a)
{
    __shared__ MutateSmem<Pol> sm;
    mutate_tile<Pol, kIndep>(a, a.iter, blockIdx.x * blockDim.x, sm);
}

// Two particles per thread (FP32 EGARCH): particles p0 + threadIdx.x and
// p0 + blockDim.x + threadIdx.x; same proposal, acceptance and outputs as
// mutate_tile, particle by particle.
template <int K, int I>
__device__ __forceinline__ void mutate_tile_x2(const MutateArgs& a, uint64_t iter, int p0,
                                               MutateSmem<PolicyEgarchF32<K, I>>& sm)
{
    using Pol = PolicyEgarchF32<K, I>;
    const int d = a.m.d;
    pdl_wait();   // as in mutate_tile
    for (int i = threadIdx.x; i < d * d; i += blockDim.x) sm.Ls[i] = a.L[i];
    if (threadIdx.x == 0) sm.acc_s = 0;
    ObsPipe<float, kChunkF32> pipe{sm.obuf, sm.bars, (const float*)a.obs, (int64_t)a.T,
                                   (a.T + kChunkF32 - 1) / kChunkF32};
    pipe.start();
    const size_t P = (size_t)a.P;
    int pq[2];
    bool act[2];
    double lpn[2];
    EgarchF32<K, I> mdl[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = p0 + h * (int)blockDim.x + (int)threadIdx.x;
        act[h] = p < a.P;
        pq[h] = act[h] ? p : a.P - 1;
        double thn[kMaxD];
        float thr[kMaxD];
        float z[kMaxD];
        proposal_normals<float>(a.seed, (uint64_t)pq[h], iter, a.cycle, d, z);
        for (int i = 0; i < d; ++i) {
            float s = 0;
            for (int k = 0; k <= i; ++k) s += sm.Ls[i * d + k] * z[k];
            thn[i] = a.theta[i * P + pq[h]] + (double)s;
            thr[i] = (float)thn[i];
            if (act[h]) a.thp[i * P + p] = thn[i];
        }
        lpn[h] = log_prior_f(a.m, thn, thr);
        float full[kMaxD];
        full_theta_f(a.m, thr, full);
        Pol::setup(mdl[h], a.m, full);
    }
    const bool ok = run_egarch_f32_x2<K, I>(mdl[0], mdl[1], pipe, a.T);
    pdl_trigger();
    if (!ok && threadIdx.x == 0) raise_error(a.err, kErrTimeout);
    unsigned int nacc = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double ll_new = ok ? mdl[h].finish(a.T) : -INFINITY;
        if (isnan(ll_new)) ll_new = -INFINITY;
        bool acc = false;
        const int p = pq[h];
        if (act[h]) {
            const double log_alpha = tempered_target(lpn[h], ll_new, a.phi) -
                                     tempered_target(a.lp[p], a.ll[p], a.phi);
            acc = mh_accept(a.seed, (uint64_t)p, iter, a.cycle, log_alpha);
            if (acc) {
                for (int i = 0; i < d; ++i) a.theta[i * P + p] = a.thp[i * P + p];
                a.ll[p] = ll_new;
                a.lp[p] = lpn[h];
                if (a.state) {
                    double st[kMaxState];
                    mdl[h].state_out(st);
                    for (int k = 0; k < Pol::kNs; ++k) a.state[k * P + p] = st[k];
                }
            }
        }
        nacc += __popc(__ballot_sync(0xffffffffu, acc));
        if (a.covtile) cov_tile_sums<Pol::kMaxFree>(a, p0 + h * (int)blockDim.x + (int)threadIdx.x, act[h]);
    }
    if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&sm.acc_s, nacc);
    __syncthreads();
    if (threadIdx.x == 0 && sm.acc_s) atomicAdd(a.acc_count, (unsigned long long)sm.acc_s);
    if (p0 == 0 && threadIdx.x == 0 && a.pending) *a.pending = 1;
    pipe.finish();
}

template <int K, int I>
__global__ void __launch_bounds__(kMutMaxThreads) k_mutate_x2(MutateArgs a)
{
    __shared__ MutateSmem<PolicyEgarchF32<K, I>> sm;
    mutate_tile_x2<K, I>(a, a.iter, blockIdx.x * 2 * blockDim.x, sm);
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

// ------------------------------------------------- data-tempering C phase
// Algorithm 1, step 2(a): w_jn(s) = w_jn(s-1) p(y_s | y_1:s-1, theta_jn) for
// s = t_l-1 + 1, ..., stopping at the first s with RSS(s) < D1 (Section 3.3),
// at a date of interest, or at T.  The search runs speculatively over a chunk
// of up to kCdataChunk observations: each block reduces, for every s of the
// chunk, (max log w, sum w, sum w^2) over its particles; one block (a warp
// per observation) combines the blocks and finds the stopping observation; a
// commit pass then
// advances every particle's recursion state, log likelihood and log weight to
// it.  The RSS statistic uses FP32 exponentials of log-weight differences; the
// log weights themselves are FP64.

struct CdataArgs {
    ModelDev m;
    const void* obs;
    int T, W;
    const double* theta;   // [d][P]
    double* state;         // [ns][P] recursion state at s0 (updated by the commit pass)
    double* ll;            // [P] log likelihood of y_1:s0 (updated by the commit pass)
    double* logw;          // [P] log weight since the cycle start (updated by the commit pass)
    int P, ns;
    int s0;                // observations already absorbed
    int B;                 // observations in this chunk (<= kCdataChunk, s0 + B <= T)
    double* part;          // [gridDim][B][3] statistics pass output
    // [1 + ns][P] (nullable): the statistics pass leaves each particle's sum
    // of the chunk's B terms and its recursion state after them, which a
    // commit of all B observations (no PIT) then takes instead of recomputing
    double* end;
    const int* stop;       // commit pass: observations to absorb (device)
    // The chunk's number within the cycle (1-based) and the device word naming
    // the chunk that holds the stop (0: none yet); a chunk numbered after it
    // does nothing, so that chunks can be queued before the stop is known.
    const int* found;
    int seq;
    int commit;
    // Commit pass, probability integral transform (Section 4.1; nullable):
    // part[block][q] gets (max log w(s-1), sum w(s-1), sum w(s-1) I[Y_s <= y_s])
    // for s = s0 + q + 1, the auxiliary draws from Philox stream `seed`.
    int pit;
    uint64_t seed;
};

// Double-float pair (value = hi + lo) for the data-tempering log weights:
// Knuth's TwoSum on the FP32 pipe.
struct Df2 {
    float hi, lo;
};

__device__ __forceinline__ Df2 df2_norm(float s, float e)
{
    const float t = s + e;
    return {t, e - (t - s)};
}

__device__ __forceinline__ Df2 df2_add_f(Df2 x, float b)
{
    const float s = x.hi + b;
    const float bv = s - x.hi;
    const float e = (x.hi - (s - bv)) + (b - bv);
    return df2_norm(s, e + x.lo);
}

__device__ __forceinline__ Df2 df2_add(Df2 x, Df2 y)
{
    const float s = x.hi + y.hi;
    const float bv = s - x.hi;
    const float e = (x.hi - (s - bv)) + (y.hi - bv);
    return df2_norm(s, e + (x.lo + y.lo));
}

// Warp maximum of normalised pairs (ordered by hi, then lo).
__device__ __forceinline__ Df2 warp_max_df2(Df2 x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, x.hi, o);
        const float l = __shfl_xor_sync(0xffffffffu, x.lo, o);
        if (h > x.hi || (h == x.hi && l > x.lo)) x = {h, l};
    }
    return x;
}

template <class Pol>
__global__ void __launch_bounds__(kMutThreads) k_cdata(CdataArgs a)
{
    using Real = typename Pol::Real;
    using Obs = typename Pol::Obs;
    __shared__ double trip[kMutThreads / 32][kCdataChunk][3];
    __shared__ float tripf[kMutThreads / 32][kCdataChunk][4];   // log2 path: warp max (hi, lo), sums
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < a.P;
    const int pp = active ? p : a.P - 1;
    const size_t P = (size_t)a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.found) {
        const int f = *a.found;
        if (f != 0 && f < a.seq) return;
    }
    if (a.commit && a.end && !a.pit && *a.stop == a.B) {
        // every observation of the chunk is absorbed: the statistics pass's
        // sum and end state are exactly what the recursion below would give
        if (active) {
            const double add = a.end[p];
            a.ll[p] += add;
            a.logw[p] += add;
            for (int k = 0; k < Pol::kNs; ++k) a.state[k * P + p] = a.end[(size_t)(1 + k) * P + p];
        }
        return;
    }
    double th[kMaxD];
    for (int i = 0; i < a.m.d; ++i) th[i] = a.theta[i * P + pp];
    typename Pol::Model mdl;
    {
        Real full[kMaxD];
        full_theta<Real>(a.m, th, full);
        Pol::setup(mdl, a.m, full);
    }
    double st[kMaxState];
    for (int k = 0; k < Pol::kNs; ++k) st[k] = a.state[k * P + pp];
    if (a.s0 > 0) Pol::load_state(mdl, st);
    double lw = a.logw[pp];
    const Obs* obs = (const Obs*)a.obs;
    if (a.commit) {
        const int n = *a.stop;
        double add = 0.0;
        if (a.pit) {
            typename Pol::Pit pm;
            Pol::pit_setup(a.m, th, pm);
            for (int q = 0; q < n; ++q) {
                const int sobs = a.s0 + q + 1;
                const double lprev = lw + add;    // log w(s-1)
                const double x = active && !isnan(lprev) ? lprev : -INFINITY;
                const double mw = warp_max(x);
                float w = 0.0f;
                if (x != -INFINITY && mw != -INFINITY) w = ex2_approx((float)((x - mw) * kLog2e));
                add += Pol::logdens(mdl, obs, sobs, a.W);
                const bool below = pm.shock(a.seed, (uint64_t)pp, sobs) <= Pol::obs_shock(mdl, obs, sobs, a.W);
                const float s1 = warp_sum(w);
                const float s2 = warp_sum(below ? w : 0.0f);
                if (lane == 0) {
                    trip[warp][q][0] = mw;
                    trip[warp][q][1] = s1;
                    trip[warp][q][2] = s2;
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                double M = -INFINITY;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, trip[w][q][0]);
                double S1 = 0.0, S2 = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    if (trip[w][q][0] == -INFINITY) continue;
                    const double e = exp(trip[w][q][0] - M);
                    S1 += trip[w][q][1] * e;
                    S2 += trip[w][q][2] * e;
                }
                double* o = a.part + ((size_t)blockIdx.x * a.B + q) * 3;
                o[0] = M;
                o[1] = S1;
                o[2] = S2;
            }
        } else if constexpr (Pol::kLog2Terms) {
            // the terms in log2 units, summed as a double-float pair on the
            // FP32 pipe (as in the statistics pass, whose sums these repeat)
            Df2 d = {0.0f, 0.0f};
            for (int q = 0; q < n; ++q) d = df2_add_f(d, Pol::logdens2(mdl, obs, a.s0 + q + 1, a.W));
            add = kLn2 * ((double)d.hi + (double)d.lo) + (double)n * Pol::kTermConst;
        } else {
            for (int q = 0; q < n; ++q) add += Pol::logdens(mdl, obs, a.s0 + q + 1, a.W);
        }
        if (isnan(add)) add = -INFINITY;
        if (active) {
            a.ll[p] += add;
            a.logw[p] = lw + add;
            if (Pol::kNs) {
                Pol::state_out(mdl, st);
                for (int k = 0; k < Pol::kNs; ++k) a.state[k * P + p] = st[k];
            }
        }
        return;
    }
    if constexpr (Pol::kLog2Terms) {
        // FP32 recursion: the log weight log w(s) = log w(s0) + sum of the
        // chunk's terms is carried in log2 units as a double-float pair (the
        // per-observation constant, common to every particle, is added back
        // to the block maxima only), so the warp maxima and the weights need no
        // FP64 instruction (each holds this part's FP64 pipe for ~64 cycles).
        const double lw2 = lw * kLog2e;
        const Df2 x0 = {(float)lw2, (float)(lw2 - (double)(float)lw2)};
        bool dead = !active || !(lw2 > -INFINITY);
        Df2 d = {0.0f, 0.0f};
        for (int q = 0; q < a.B; ++q) {
            const float u = Pol::logdens2(mdl, obs, a.s0 + q + 1, a.W);
            dead = dead || !(u > -INFINITY && u < INFINITY);
            d = df2_add_f(d, u);
            const Df2 x = dead ? Df2{-INFINITY, 0.0f} : df2_add(x0, d);
            const Df2 mx = warp_max_df2(x);
            float w = 0.0f;
            if (!dead && mx.hi != -INFINITY) w = ex2_approx((x.hi - mx.hi) + (x.lo - mx.lo));
            const float s1 = warp_sum(w);
            const float s2 = warp_sum(w * w);
            if (lane == 0) {
                tripf[warp][q][0] = mx.hi;
                tripf[warp][q][1] = mx.lo;
                tripf[warp][q][2] = s1;
                tripf[warp][q][3] = s2;
            }
        }
        if (a.end && active) {   // the commit pass's sum over all B terms
            double add = kLn2 * ((double)d.hi + (double)d.lo) + (double)a.B * Pol::kTermConst;
            if (isnan(add)) add = -INFINITY;
            a.end[p] = add;
        }
    } else {
        double add = 0.0;   // the commit pass's sum, in its order
        for (int q = 0; q < a.B; ++q) {
            double l = Pol::logdens(mdl, obs, a.s0 + q + 1, a.W);
            add += l;
            lw += isnan(l) ? -INFINITY : l;
            const double x = active ? lw : -INFINITY;
            const double mw = warp_max(x);
            float w = 0.0f;
            if (x != -INFINITY && mw != -INFINITY) w = ex2_approx((float)((x - mw) * kLog2e));
            const float s1 = warp_sum(w);
            const float s2 = warp_sum(w * w);
            if (lane == 0) {
                trip[warp][q][0] = mw;
                trip[warp][q][1] = s1;
                trip[warp][q][2] = s2;
            }
        }
        if (a.end && active) a.end[p] = isnan(add) ? -INFINITY : add;
    }
    if (a.end && active && Pol::kNs) {
        Pol::state_out(mdl, st);
        for (int k = 0; k < Pol::kNs; ++k) a.end[(size_t)(1 + k) * P + p] = st[k];
    }
    __syncthreads();
    if constexpr (Pol::kLog2Terms) {
        // the warps' (max, sums) in log2 units combined on the FP32 pipe; one
        // conversion to natural units (with the per-observation constant) per
        // observation
        for (int q = threadIdx.x; q < a.B; q += blockDim.x) {
            Df2 M = {-INFINITY, 0.0f};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const float h = tripf[w][q][0], l = tripf[w][q][1];
                if (h > M.hi || (h == M.hi && l > M.lo)) M = {h, l};
            }
            Df2 S1 = {0.0f, 0.0f}, S2 = {0.0f, 0.0f};
            if (M.hi != -INFINITY)
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    if (tripf[w][q][0] == -INFINITY) continue;
                    const float e = ex2_approx((tripf[w][q][0] - M.hi) + (tripf[w][q][1] - M.lo));
                    S1 = df2_add_f(S1, tripf[w][q][2] * e);
                    S2 = df2_add_f(S2, tripf[w][q][3] * (e * e));
                }
            double* o = a.part + ((size_t)blockIdx.x * a.B + q) * 3;
            o[0] = M.hi == -INFINITY ? -INFINITY
                                     : kLn2 * ((double)M.hi + (double)M.lo) + (double)(q + 1) * Pol::kTermConst;
            o[1] = (double)S1.hi + (double)S1.lo;
            o[2] = (double)S2.hi + (double)S2.lo;
        }
    } else {
        for (int q = threadIdx.x; q < a.B; q += blockDim.x) {
            double M = -INFINITY;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, trip[w][q][0]);
            // the warps' sums rescaled by FP32 exponentials of the FP64 differences
            // (the sums are of FP32 weights already)
            double S1 = 0.0, S2 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                if (trip[w][q][0] == -INFINITY) continue;
                const float e = ex2_approx((float)(trip[w][q][0] - M) * (float)kLog2e);
                S1 += trip[w][q][1] * (double)e;
                S2 += trip[w][q][2] * (double)(e * e);
            }
            double* o = a.part + ((size_t)blockIdx.x * a.B + q) * 3;
            o[0] = M;
            o[1] = S1;
            o[2] = S2;
        }
    }
}

// Host-side launchers (defined in the instantiation units).
// lq[p] = -|L^{-1}(theta_p - qmean)|^2 / 2 by forward substitution in FP64, a
// zero pivot contributing nothing (defined in phase.cu).
cudaError_t launch_indep_logq(const double* theta, int d, int P, const double* L, const double* qmean,
                              double* lq, cudaStream_t s);
cudaError_t launch_mutate(const MutateArgs& a, int precision, int threads, cudaStream_t s);
cudaError_t launch_loglik(const LoglikArgs& a, int precision, cudaStream_t s);
cudaError_t launch_cdata(const CdataArgs& a, int precision, cudaStream_t s);

}  // namespace smc
