// Host driver and C ABI (include/smc.h).
//
// The driver runs Algorithm 2 with the Section 3.3 specifics on one GPU.  All
// particle data stay on the device; a cycle enqueues its kernels on the
// context's stream and reads back one small control block after the C/S
// phases (the power reached, RSS) and one after the M phase (acceptance), so
// the host decides the number of Metropolis iterations exactly as the paper's
// rules state.

#include "ctx.h"

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace smc {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

#define SMC_DECL_EGARCH(TAG, K)                                                 \
    cudaError_t launch_mutate_##TAG##_k##K(const MutateArgs& a, int threads, cudaStream_t s); \
    cudaError_t launch_loglik_##TAG##_k##K(const LoglikArgs& a, cudaStream_t s);
SMC_DECL_EGARCH(f32, 1)
SMC_DECL_EGARCH(f32, 2)
SMC_DECL_EGARCH(f32, 3)
SMC_DECL_EGARCH(f32, 4)
SMC_DECL_EGARCH(f64, 1)
SMC_DECL_EGARCH(f64, 2)
SMC_DECL_EGARCH(f64, 3)
SMC_DECL_EGARCH(f64, 4)
cudaError_t launch_mutate_linreg(const MutateArgs& a, int threads, cudaStream_t s);
cudaError_t launch_loglik_linreg(const LoglikArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f32_k1(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f32_k2(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f32_k3(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f32_k4(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f64_k1(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f64_k2(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f64_k3(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_f64_k4(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_cdata_linreg(const CdataArgs& a, cudaStream_t s);
cudaError_t launch_mutate_x2_f32_k1(const MutateArgs& a, int threads, cudaStream_t s);
cudaError_t launch_mutate_x2_f32_k2(const MutateArgs& a, int threads, cudaStream_t s);
cudaError_t launch_mutate_x2_f32_k3(const MutateArgs& a, int threads, cudaStream_t s);
cudaError_t launch_mutate_x2_f32_k4(const MutateArgs& a, int threads, cudaStream_t s);

static bool valid_mut_threads(int t) { return t >= 32 && t <= kMutMaxThreads && t % 32 == 0; }

// Block size that spreads P particles (ppt per thread) most evenly over the
// SMs: the fewest blocks per SM k for which ceil(warps / (SMs k)) warps fit in
// one block.  At 65,536 particles, two per thread, on 152 SMs: 7 warps, one
// block per SM, where 64-thread blocks leave 56 SMs with 8 warps and 96 with 6.
static int balanced_threads(int P, int ppt)
{
    const int warps = (P + 32 * ppt - 1) / (32 * ppt);
    const int sms = device_sm_count();
    for (int k = 1; k <= 64; ++k) {
        const int b = (warps + sms * k - 1) / (sms * k);
        if (b <= kMutMaxThreads / 32) return 32 * b;
    }
    return kMutMaxThreads;
}

cudaError_t launch_mutate_x2(const MutateArgs& a, int threads, cudaStream_t s)
{
    if (a.qmean || !valid_mut_threads(threads)) return cudaErrorInvalidValue;   // random walk only
    count_launch();
    switch (a.m.K) {
    case 1: return launch_mutate_x2_f32_k1(a, threads, s);
    case 2: return launch_mutate_x2_f32_k2(a, threads, s);
    case 3: return launch_mutate_x2_f32_k3(a, threads, s);
    case 4: return launch_mutate_x2_f32_k4(a, threads, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cdata(const CdataArgs& a, int precision, cudaStream_t s)
{
    count_launch();
    if (a.m.kind == SMC_LINREG) return launch_cdata_linreg(a, s);
    if (precision == SMC_FP32) {
        switch (a.m.K) {
        case 1: return launch_cdata_f32_k1(a, s);
        case 2: return launch_cdata_f32_k2(a, s);
        case 3: return launch_cdata_f32_k3(a, s);
        case 4: return launch_cdata_f32_k4(a, s);
        }
    } else {
        switch (a.m.K) {
        case 1: return launch_cdata_f64_k1(a, s);
        case 2: return launch_cdata_f64_k2(a, s);
        case 3: return launch_cdata_f64_k3(a, s);
        case 4: return launch_cdata_f64_k4(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mutate(const MutateArgs& a, int precision, int threads, cudaStream_t s)
{
    count_launch();
    if (!valid_mut_threads(threads)) return cudaErrorInvalidValue;
    if (a.m.kind == SMC_LINREG) return launch_mutate_linreg(a, threads, s);
    if (precision == SMC_FP32) {
        switch (a.m.K) {
        case 1: return launch_mutate_f32_k1(a, threads, s);
        case 2: return launch_mutate_f32_k2(a, threads, s);
        case 3: return launch_mutate_f32_k3(a, threads, s);
        case 4: return launch_mutate_f32_k4(a, threads, s);
        }
    } else {
        switch (a.m.K) {
        case 1: return launch_mutate_f64_k1(a, threads, s);
        case 2: return launch_mutate_f64_k2(a, threads, s);
        case 3: return launch_mutate_f64_k3(a, threads, s);
        case 4: return launch_mutate_f64_k4(a, threads, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_loglik(const LoglikArgs& a, int precision, cudaStream_t s)
{
    count_launch();
    if (a.m.kind == SMC_LINREG) return launch_loglik_linreg(a, s);
    if (precision == SMC_FP32) {
        switch (a.m.K) {
        case 1: return launch_loglik_f32_k1(a, s);
        case 2: return launch_loglik_f32_k2(a, s);
        case 3: return launch_loglik_f32_k3(a, s);
        case 4: return launch_loglik_f32_k4(a, s);
        }
    } else {
        switch (a.m.K) {
        case 1: return launch_loglik_f64_k1(a, s);
        case 2: return launch_loglik_f64_k2(a, s);
        case 3: return launch_loglik_f64_k3(a, s);
        case 4: return launch_loglik_f64_k4(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ small kernels
// Particle-major [P][d] -> parameter-major [d][P].
__global__ void k_to_soa(const double* __restrict__ in, int P, int d, double* __restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)P * d) return;
    const size_t p = e / d, i = e % d;
    out[i * (size_t)P + p] = in[e];
}

__global__ void k_to_aos(const double* __restrict__ in, int P, int d, double* __restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)P * d) return;
    const size_t p = e / d, i = e % d;
    out[e] = in[i * (size_t)P + p];
}

__global__ void k_f64_to_f32(const double* __restrict__ in, size_t n, float* __restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (float)in[e];
}

// Data tempering start: log prior of the prior draws, empty-sample likelihood
// and volatility state at v_k0 = 0.
__global__ void k_init_data_tempering(ModelDev m, const double* __restrict__ theta, int P, int ns,
                                      double* ll, double* lp, double* state)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double th[kMaxD];
    for (int i = 0; i < m.d; ++i) th[i] = theta[i * (size_t)P + p];
    lp[p] = log_prior(m, th);
    ll[p] = 0.0;
    for (int k = 0; k < ns; ++k) state[k * (size_t)P + p] = 0.0;
}

}  // namespace smc

using namespace smc;

static smc_status set_err(smc_ctx* c, smc_status st, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_err(ctx, SMC_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                           __FILE__, __LINE__);                                               \
    } while (0)

static void fill_model_dev(const smc_model& m, ModelDev& d)
{
    std::memset(&d, 0, sizeof d);
    d.kind = m.model;
    d.K = m.K;
    d.I = m.I;
    d.gamma = m.gamma;
    d.eps0_zero = m.eps0_zero;
    d.p = m.p;
    d.sigma = m.sigma;
    d.d_full = m.d_full;
    d.d = m.n_free > 0 ? m.n_free : m.d_full;
    d.has_free = m.n_free > 0;
    for (int i = 0; i < SMC_MAX_D; ++i) {
        d.free_idx[i] = m.free_idx[i];
        d.theta_fixed[i] = m.theta_fixed[i];
        d.prior_mean[i] = m.prior_mean[i];
        const double sd = m.prior_sd[i] > 0.0 ? m.prior_sd[i] : 1.0;
        d.prior_isd[i] = 1.0 / sd;
        d.prior_c[i] = -0.5 * kLog2Pi - std::log(sd);
        d.prior_lo[i] = m.prior_lo[i];
        d.prior_mean_f[i] = (float)d.prior_mean[i];
        d.prior_isd_f[i] = (float)d.prior_isd[i];
        d.prior_c_f[i] = (float)d.prior_c[i];
        d.prior_lo_f[i] = (float)d.prior_lo[i];
    }
}

static smc_status validate_model(const smc_model* m, smc_ctx* ctx)
{
    if (!m) return set_err(ctx, SMC_EINVAL, "model is NULL");
    if (m->model == SMC_EGARCH) {
        if (m->K < 1 || m->K > kMaxK || m->I < 1 || m->I > kMaxI)
            return set_err(ctx, SMC_EINVAL, "EGARCH needs 1 <= K <= %d and 1 <= I <= %d", kMaxK, kMaxI);
    } else if (m->model == SMC_LINREG) {
        if (m->p < 1 || m->p > 7 || !(m->sigma > 0.0))
            return set_err(ctx, SMC_EINVAL, "LINREG needs 1 <= p <= 7 and sigma > 0");
    } else {
        return set_err(ctx, SMC_EINVAL, "unknown model %d", m->model);
    }
    if (m->d_full < 1 || m->d_full > SMC_MAX_D) return set_err(ctx, SMC_EINVAL, "bad d_full %d", m->d_full);
    if (m->n_free < 0 || m->n_free > m->d_full) return set_err(ctx, SMC_EINVAL, "bad n_free %d", m->n_free);
    const int d = m->n_free > 0 ? m->n_free : m->d_full;
    for (int i = 0; i < m->n_free; ++i)
        if (m->free_idx[i] < 0 || m->free_idx[i] >= m->d_full)
            return set_err(ctx, SMC_EINVAL, "free_idx[%d] out of range", i);
    for (int i = 0; i < d; ++i)
        if (!(m->prior_sd[i] > 0.0) || !std::isfinite(m->prior_mean[i]))
            return set_err(ctx, SMC_EINVAL, "prior %d invalid", i);
    return SMC_OK;
}

extern "C" {

smc_status smc_model_egarch(smc_model* m, int K, int I, int gamma)
{
    if (!m || K < 1 || K > kMaxK || I < 1 || I > kMaxI) return SMC_EINVAL;
    std::memset(m, 0, sizeof *m);
    m->model = SMC_EGARCH;
    m->K = K;
    m->I = I;
    m->gamma = gamma ? 1 : 0;
    int j = 0;
    auto put = [&](double mean, double sd, double lo) {
        m->prior_mean[j] = mean;
        m->prior_sd[j] = sd;
        m->prior_lo[j] = lo;
        ++j;
    };
    // Table 1 (Section 5.1).
    put(0.0, 1.0, -INFINITY);                                      // theta_1
    put(std::log(0.01), 1.0, -INFINITY);                           // theta_2
    for (int k = 0; k < K; ++k) put(std::atanh(0.95), 1.0, -INFINITY);   // theta_3k
    for (int k = 0; k < K; ++k) put(std::log(0.10), 1.0, -INFINITY);     // theta_4k
    if (gamma)
        for (int k = 0; k < K; ++k) put(0.0, 0.2, -INFINITY);      // theta_5k
    if (I >= 2) {
        for (int i = 0; i < I; ++i) put(0.0, 1.0, -INFINITY);      // theta_6i
        for (int i = 0; i < I; ++i) put(0.0, 1.0, -INFINITY);      // theta_7i
        for (int i = 0; i < I; ++i) put(0.0, 1.0, -3.0);           // theta_8i
    }
    m->d_full = j;
    return SMC_OK;
}

int smc_linreg_width(int p) { return p + 1 <= 2 ? 2 : (p + 1 <= 4 ? 4 : 8); }

smc_status smc_model_linreg(smc_model* m, int p, double sigma, const double* prior_mean,
                            const double* prior_sd)
{
    if (!m || p < 1 || p > 7 || !(sigma > 0.0) || !prior_mean || !prior_sd) return SMC_EINVAL;
    std::memset(m, 0, sizeof *m);
    m->model = SMC_LINREG;
    m->p = p;
    m->sigma = sigma;
    m->d_full = p;
    for (int i = 0; i < p; ++i) {
        m->prior_mean[i] = prior_mean[i];
        m->prior_sd[i] = prior_sd[i];
        m->prior_lo[i] = -INFINITY;
    }
    return SMC_OK;
}

int smc_model_dim(const smc_model* m) { return m ? (m->n_free > 0 ? m->n_free : m->d_full) : 0; }

void smc_config_default(smc_config* c)
{
    std::memset(c, 0, sizeof *c);
    c->J = 64;
    c->N = 1024;
    c->precision = SMC_FP32;
    c->tempering = SMC_POWER;
    c->mutation = SMC_RW;
    c->resampler = SMC_RESIDUAL;
    c->d1 = 0.5;
    c->d2 = 0.2;
    c->stop_rule = SMC_STOP_DET;
    c->rbar = 7;
    c->kappa = 3;
    c->rmax = 100;
    c->e1 = 0.35;
    c->e2 = 0.90;
    c->h0_tenths = 5;
    c->hmin_tenths = 1;
    c->hmax_tenths = 10;
    c->acc_target = 0.25;
    c->h_reset_each_cycle = 0;
    c->n_force = 0;
    c->search_passes = 6;
    c->seed = 1;
    c->burnin = 0;
    c->pit = 0;
}

uint64_t smc_launch_count(void) { return g_launches.load(); }

const char* smc_status_str(smc_status s)
{
    switch (s) {
    case SMC_OK: return "ok";
    case SMC_EINVAL: return "invalid argument";
    case SMC_ENOMEM: return "out of memory";
    case SMC_ECUDA: return "CUDA error";
    case SMC_EDEGENERATE: return "degenerate weights";
    case SMC_ENONFINITE: return "non-finite input";
    case SMC_ETIMEOUT: return "device wait timed out";
    case SMC_EDONE: return "run complete";
    }
    return "unknown status";
}

const char* smc_last_error(const smc_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

}  // extern "C"

// ------------------------------------------------------------- helpers
static void release(smc_ctx* c)
{
    if (!c) return;
    void* ptrs[] = {c->obs, c->theta[0], c->theta[1], c->ll[0], c->ll[1], c->lp[0], c->lp[1],
                    c->grad[0], c->grad[1], c->ckpt, c->design_L,
                    c->state[0], c->state[1], c->thp, c->logw, c->g, c->a, c->lw, c->gstat,
                    c->idx, c->cov_part, c->search_part, c->cd_part, c->cd_end, c->mom_part, c->mom_out, c->ml_out,
                    c->L, c->qmean, c->covtile, c->covshift_f, c->cov_tot, c->cov_counter, c->lq, c->a_score, c->pit, c->gather_ptrs, c->ctl};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    for (auto& e : c->ev_pool) cudaEventDestroy(e);
    for (auto& pr : c->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

static smc_status check_device_error(smc_ctx* ctx, const Ctl& h)
{
    if (h.err & kErrTimeout) return set_err(ctx, SMC_ETIMEOUT, "a bounded device wait ran out");
    if (h.err & kErrDegenerate) return set_err(ctx, SMC_EDEGENERATE, "a group has zero total weight");
    if (h.err & kErrBounds) return set_err(ctx, SMC_ECUDA, "internal index check failed");
    return SMC_OK;
}

static smc_status check_device_error(smc_ctx* ctx) { return check_device_error(ctx, *ctx->ctl_host); }

static smc_status sync_ctl(smc_ctx* ctx)
{
    CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->d2h += sizeof(Ctl);
    CU(cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

static smc_status fold_profile(smc_ctx* ctx)
{
    for (auto& pr : ctx->ev_pending) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, pr.first, pr.second));
        ctx->mutate_ms += ms;
        ctx->ev_pool.push_back(pr.first);
        ctx->ev_pool.push_back(pr.second);
    }
    ctx->ev_pending.clear();
    return SMC_OK;
}

static cudaEvent_t take_event(smc_ctx* ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// One M-phase Metropolis iteration: covariance + Cholesky (with the pending h
// update), then the fused proposal/likelihood/accept kernel.
static smc_status m_iteration(smc_ctx* ctx, int r, int Tm, double phi)
{
    const smc_config& c = ctx->cfg;
    const int P = ctx->P, d = ctx->d;
    double* th = ctx->theta[ctx->cur];
    const size_t dd = (size_t)d * d;
    if (ctx->replay) {
        if (ctx->replay_iter >= ctx->design_iters)
            return set_err(ctx, SMC_EINVAL, "the replayed design has only %d iterations", ctx->design_iters);
        CU(cudaMemcpyAsync(ctx->L, ctx->design_L + (size_t)ctx->replay_iter * dd, dd * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream));
        ctx->replay_iter += 1;
    } else {
        // Sigma = h^2 V; the independent sampler takes V itself (h pinned at
        // 10 tenths for the factor, still updated from the acceptance rate)
        // and the pooled mean.
        // The S phase's gather (first iteration) or the previous mutation
        // launch has left the covariance tile sums of the current particles.
        const bool indep = c.mutation == SMC_INDEP;
        if (ctx->tiles_ready)
            CU(launch_cov_tiles(ctx->covtile, ctx->ntiles, ctx->tile_kd, d, P, ctx->cov_tot, ctx->cov_counter,
                                ctx->covshift_f, ctx->qmean, ctx->ctl, indep ? 10 : 0, c.acc_target,
                                c.hmin_tenths, c.hmax_tenths, ctx->L, ctx->stream));
        else
            CU(launch_cov(th, d, P, ctx->cov_part, ctx->cov_G, ctx->cov_counter, ctx->ctl, indep ? 10 : 0,
                          c.acc_target, c.hmin_tenths, c.hmax_tenths, ctx->qmean, nullptr, ctx->L,
                          ctx->stream, ctx->covshift_f));
        if (indep) CU(launch_indep_logq(th, d, P, ctx->L, ctx->qmean, ctx->lq, ctx->stream));
    }
    if (ctx->record) {
        if (ctx->design_iters >= ctx->design_cap)
            return set_err(ctx, SMC_ENOMEM, "design record is full (%d iterations)", ctx->design_cap);
        CU(cudaMemcpyAsync(ctx->design_L + (size_t)ctx->design_iters * dd, ctx->L, dd * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream));
        ctx->design_iters += 1;
    }
    if (c.mutation == SMC_MALA) {
        MalaArgs a;
        a.m = ctx->mdev;
        a.obs = ctx->obs;
        a.T = Tm;
        a.W = ctx->W;
        a.theta = th;
        a.ll = ctx->ll[ctx->cur];
        a.lp = ctx->lp[ctx->cur];
        a.state = ctx->ns ? ctx->state[ctx->cur] : nullptr;
        a.grad = ctx->grad[ctx->cur];
        a.ckpt = ctx->ckpt;
        a.P = P;
        a.ns = ctx->ns;
        a.L = ctx->L;
        a.phi = phi;
        a.seed = c.seed;
        a.cycle = (uint64_t)ctx->cycle;
        a.iter = (uint64_t)r;
        a.acc_count = &ctx->ctl->acc_count;
        a.pending = &ctx->ctl->pending;
        a.err = &ctx->ctl->err;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const bool timed = ctx->profile == 1 || (ctx->profile == 2 && r == 0);
        if (timed) {
            e0 = take_event(ctx);
            e1 = take_event(ctx);
            CU(cudaEventRecord(e0, ctx->stream));
        }
        CU(launch_mala(a, c.precision, ctx->stream));
        if (timed) {
            CU(cudaEventRecord(e1, ctx->stream));
            ctx->ev_pending.push_back({e0, e1});
            ctx->mutate_launches += 1;
        }
        return SMC_OK;
    }
    MutateArgs a;
    a.m = ctx->mdev;
    a.obs = ctx->obs;
    a.T = Tm;
    a.W = ctx->W;
    a.theta = th;
    a.ll = ctx->ll[ctx->cur];
    a.lp = ctx->lp[ctx->cur];
    a.state = ctx->ns ? ctx->state[ctx->cur] : nullptr;
    a.thp = ctx->thp;
    a.P = P;
    a.ns = ctx->ns;
    a.L = ctx->L;
    a.qmean = c.mutation == SMC_INDEP ? ctx->qmean : nullptr;
    a.lq = ctx->lq;
    const bool tiles = ctx->covtile && !ctx->replay;
    a.covtile = tiles ? ctx->covtile : nullptr;
    a.covshift = ctx->covshift_f;
    a.ntiles = ctx->ntiles;
    ctx->tiles_ready = tiles;
    a.phi = phi;
    a.seed = c.seed;
    a.cycle = (uint64_t)ctx->cycle;
    a.iter = (uint64_t)r;
    a.acc_count = &ctx->ctl->acc_count;
    a.pending = &ctx->ctl->pending;
    a.err = &ctx->ctl->err;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = ctx->profile == 1 || (ctx->profile == 2 && r == 0);
    // a timed launch sits between two events, which serialise it anyway: it is
    // launched plainly so that the events bracket the kernel alone
    a.dependent = timed ? 0 : 1;
    if (timed) {
        e0 = take_event(ctx);
        e1 = take_event(ctx);
        CU(cudaEventRecord(e0, ctx->stream));
    }
    if (ctx->ppt == 2) CU(launch_mutate_x2(a, ctx->mut_threads, ctx->stream));
    else CU(launch_mutate(a, c.precision, ctx->mut_threads, ctx->stream));
    if (timed) {
        CU(cudaEventRecord(e1, ctx->stream));
        ctx->ev_pending.push_back({e0, e1});
        ctx->mutate_launches += 1;
    }
    return SMC_OK;
}

// MALA: log likelihood and its gradient of the current particles over y_1:T.
static smc_status refresh_gradient(smc_ctx* ctx, int T)
{
    GradArgs g;
    g.m = ctx->mdev;
    g.obs = ctx->obs;
    g.T = T;
    g.W = ctx->W;
    g.theta = ctx->theta[ctx->cur];
    g.P = ctx->P;
    g.ll = ctx->ll[ctx->cur];
    g.grad = ctx->grad[ctx->cur];
    g.state = ctx->ns ? ctx->state[ctx->cur] : nullptr;
    g.ckpt = ctx->ckpt;
    CU(launch_loglik_grad(g, ctx->cfg.precision, ctx->stream));
    return SMC_OK;
}

static smc_status test_functions(smc_ctx* ctx, int rne_only)
{
    // EGARCH: g1..g3 rows; other models: the parameters themselves.
    const int P = ctx->P;
    if (ctx->model.model == SMC_EGARCH) {
        CU(launch_testfn(ctx->mdev, ctx->cfg.precision, ctx->theta[ctx->cur], ctx->state[ctx->cur], P,
                         ctx->g, ctx->stream));
        CU(launch_moments(ctx->g, 3, ctx->cfg.J, ctx->cfg.N, ctx->mom_part, ctx->mom_out, ctx->ctl, 0,
                          ctx->stream));
    } else {
        CU(launch_moments(ctx->theta[ctx->cur], ctx->d, ctx->cfg.J, ctx->cfg.N, ctx->mom_part,
                          ctx->mom_out, ctx->ctl, 0, ctx->stream));
    }
    (void)rne_only;
    return SMC_OK;
}

// S phase (resampling within groups + gather into the other buffer set).
static smc_status s_phase(smc_ctx* ctx, int mode)
{
    const smc_config& c = ctx->cfg;
    SelectArgs s;
    std::memset(&s, 0, sizeof s);
    s.mode = mode;
    s.ll = ctx->ll[ctx->cur];
    s.logw = ctx->logw;
    s.J = c.J;
    s.N = c.N;
    s.scheme = c.resampler;
    s.seed = c.seed;
    s.cycle = (uint64_t)ctx->cycle;
    s.a = ctx->a;
    s.a_score = c.burnin > 0 && c.tempering == SMC_DATA && ctx->t_prev >= c.burnin ? ctx->a_score : nullptr;
    s.lw = ctx->lw;
    s.gstat = ctx->gstat;
    s.idx = ctx->idx;
    s.ctl = ctx->ctl;
    s.err = &ctx->ctl->err;
    CU(launch_select(s, ctx->stream));
    GatherArgs g;
    g.idx = ctx->idx;
    g.N = c.N;
    g.P = ctx->P;
    g.nrows = ctx->gather_rows;
    g.src = ctx->gather_ptrs + (size_t)ctx->cur * ctx->gather_rows * 2;
    g.dst = ctx->gather_ptrs + (size_t)ctx->cur * ctx->gather_rows * 2 + ctx->gather_rows;
    // the next M phase's first covariance step takes its sums from the gather
    const bool tiles = ctx->covtile && !ctx->replay;
    g.covtile = tiles ? ctx->covtile : nullptr;
    g.covshift = ctx->covshift_f;
    g.ntiles = ctx->ntiles;
    g.d = ctx->d;
    g.tile_kd = ctx->tile_kd;
    CU(launch_gather(g, ctx->stream));
    ctx->tiles_ready = tiles;
    ctx->cur ^= 1;
    return SMC_OK;
}

static smc_status start_run(smc_ctx* ctx, const double* theta0, int theta0_on_device);

// ------------------------------------------------------------ driver steps
smc_status smc_internal_enqueue_cs(smc_ctx* ctx)
{
    const smc_config& c = ctx->cfg;
    ctx->cycle += 1;
    if (ctx->replay) {
        // C phase of Algorithm 1 with the recorded schedule
        if (ctx->cycle > (int)ctx->design_x.size())
            return set_err(ctx, SMC_EINVAL, "the replayed design has only %d cycles", (int)ctx->design_x.size());
        CU(launch_set_power(ctx->ctl, ctx->design_x[ctx->cycle - 1], ctx->stream));
    } else {
        // C phase: next power by k-ary bisection on RSS
        CU(launch_power_search(ctx->ll[ctx->cur], ctx->P, c.d1, c.search_passes, ctx->search_part, ctx->ctl,
                               ctx->stream));
    }
    // S phase (weights dphi * l_n), then pooled RSS, log wtilde and phi
    smc_status st = s_phase(ctx, 0);
    if (st != SMC_OK) return st;
    CU(launch_cycle_close(ctx->gstat, ctx->lw, c.J, c.N, 1, ctx->ctl, ctx->stream));
    return SMC_OK;
}

smc_status smc_internal_enqueue_ctl_readback(smc_ctx* ctx)
{
    CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->d2h += sizeof(Ctl);
    return SMC_OK;
}

smc_status smc_internal_check(smc_ctx* ctx) { return check_device_error(ctx); }

void smc_internal_after_cs(smc_ctx* ctx, double* rss, int* forced)
{
    ctx->phi = ctx->ctl_host->phi;
    *rss = ctx->ctl_host->rss;
    *forced = ctx->ctl_host->last;
}

int smc_internal_R(const smc_ctx* ctx, double rss)
{
    const smc_config& c = ctx->cfg;
    return c.stop_rule == SMC_STOP_DET ? (rss < c.d2 ? c.kappa * c.rbar : c.rbar) : c.rmax;
}

smc_status smc_internal_enqueue_adapt(smc_ctx* ctx)
{
    const smc_config& c = ctx->cfg;
    CU(launch_adapt_h(ctx->ctl, ctx->P, c.acc_target, c.hmin_tenths, c.hmax_tenths, ctx->stream));
    return SMC_OK;
}

// Host bookkeeping at the end of an M phase from the control block h read
// back after it; `cycle` is the cycle that ends.
static smc_status after_m_from(smc_ctx* ctx, const Ctl& h, int cycle, int t_l, int R, int Tm, double phim,
                               double rss, smc_cycle_info* info)
{
    const smc_config& c = ctx->cfg;
    const int P = ctx->P;
    if (ctx->profile) {
        smc_status st = fold_profile(ctx);
        if (st != SMC_OK) return st;
    }
    if (ctx->record) {
        ctx->design_x.push_back(c.tempering == SMC_POWER ? h.phi : (double)t_l);
        ctx->design_R.push_back(R);
    }
    ctx->t_prev = t_l;
    ctx->msteps += R;
    ctx->evals += (double)R * (double)P * (double)Tm;
    if (c.tempering == SMC_POWER ? h.last : (t_l >= ctx->T)) ctx->done = 1;
    if (info) {
        info->cycle = cycle;
        info->t = t_l;
        info->phi = phim;
        info->rss = rss;
        info->R = R;
        info->h_tenths = h.h_tenths;
        info->acc_rate = h.acc_n ? h.acc_sum / h.acc_n : 0.0;
        info->evals = (double)R * (double)P * (double)Tm;
        info->done = ctx->done;
    }
    return SMC_OK;
}

smc_status smc_internal_after_m(smc_ctx* ctx, int t_l, int R, int Tm, double phim, double rss,
                                smc_cycle_info* info)
{
    return after_m_from(ctx, *ctx->ctl_host, ctx->cycle, t_l, R, Tm, phim, rss, info);
}

extern "C" {

smc_status smc_init(const smc_model* m, const smc_config* c, const double* y, const double* X,
                    int T, const double* theta0, int theta0_on_device, void* stream, smc_ctx** out)
{
    if (!out) return SMC_EINVAL;
    *out = nullptr;
    smc_ctx* ctx = new (std::nothrow) smc_ctx();
    if (!ctx) return SMC_ENOMEM;
    *out = ctx;   // caller frees even on error, so the message stays readable
    smc_status st = validate_model(m, ctx);
    if (st != SMC_OK) return st;
    if (!c) return set_err(ctx, SMC_EINVAL, "config is NULL");
    if (c->J < 2 || c->N < 1 || c->N > SMC_MAX_N)
        return set_err(ctx, SMC_EINVAL, "need J >= 2 and 1 <= N <= %d", SMC_MAX_N);
    if ((long long)c->J * c->N > (1ll << 30)) return set_err(ctx, SMC_EINVAL, "too many particles");
    if (T < 1 || !y) return set_err(ctx, SMC_EINVAL, "need T >= 1 observations");
    if (m->model == SMC_LINREG && !X) return set_err(ctx, SMC_EINVAL, "LINREG needs X");
    if (!theta0) return set_err(ctx, SMC_EINVAL, "theta0 is NULL");
    if (c->mutation != SMC_RW && c->mutation != SMC_MALA && c->mutation != SMC_INDEP)
        return set_err(ctx, SMC_EINVAL, "unknown mutation %d", c->mutation);
    if (c->tempering != SMC_POWER && c->tempering != SMC_DATA)
        return set_err(ctx, SMC_EINVAL, "unknown tempering %d", c->tempering);
    if (c->precision != SMC_FP32 && c->precision != SMC_FP64)
        return set_err(ctx, SMC_EINVAL, "unknown precision %d", c->precision);
    if (m->model == SMC_LINREG && c->precision != SMC_FP64)
        return set_err(ctx, SMC_EINVAL, "LINREG runs in FP64 only");
    if (!(c->d1 > 0.0 && c->d1 < 1.0) || c->rbar < 1 || c->kappa < 1 || c->rmax < 1 ||
        c->hmin_tenths < 1 || c->hmax_tenths < c->hmin_tenths || c->h0_tenths < c->hmin_tenths ||
        c->h0_tenths > c->hmax_tenths || c->search_passes < 1 || c->n_force < 0 ||
        c->n_force > SMC_MAX_FORCE)
        return set_err(ctx, SMC_EINVAL, "invalid simulator settings");
    if ((c->burnin != 0 || c->pit != 0) && c->tempering != SMC_DATA)
        return set_err(ctx, SMC_EINVAL, "the log score and the PIT need data tempering");
    if (c->burnin < 0 || c->burnin >= T || (c->pit != 0 && c->pit != 1))
        return set_err(ctx, SMC_EINVAL, "need 0 <= burnin < T and pit in {0, 1}");
    for (int t = 0; t < T; ++t)
        if (!std::isfinite(y[t])) return set_err(ctx, SMC_ENONFINITE, "y[%d] is not finite", t);
    if (X)
        for (long long i = 0; i < (long long)T * m->p; ++i)
            if (!std::isfinite(X[i])) return set_err(ctx, SMC_ENONFINITE, "X[%lld] is not finite", i);

    ctx->model = *m;
    ctx->cfg = *c;
    fill_model_dev(*m, ctx->mdev);
    ctx->T = T;
    ctx->P = c->J * c->N;
    ctx->d = ctx->mdev.d;
    ctx->ns = m->model == SMC_EGARCH ? m->K + 1 : 0;
    ctx->W = m->model == SMC_LINREG ? smc_linreg_width(m->p) : 1;
    ctx->stream = (cudaStream_t)stream;
    const int P = ctx->P, d = ctx->d, J = c->J;
    const size_t Ps = (size_t)P;

    // observations
    if (m->model == SMC_LINREG) {
        std::vector<double> rec((size_t)T * ctx->W, 0.0);
        for (int t = 0; t < T; ++t) {
            for (int i = 0; i < m->p; ++i) rec[(size_t)t * ctx->W + i] = X[(size_t)t * m->p + i];
            rec[(size_t)t * ctx->W + m->p] = y[t];
        }
        double* o;
        CU(dalloc(&o, rec.size()));
        ctx->obs = o;
        CU(cudaMemcpyAsync(o, rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        ctx->h2d += rec.size() * sizeof(double);
        CU(cudaStreamSynchronize(ctx->stream));
    } else if (c->precision == SMC_FP32) {
        double* tmp;
        float* o;
        CU(dalloc(&tmp, T));
        CU(dalloc(&o, T));
        ctx->obs = o;
        CU(cudaMemcpyAsync(tmp, y, (size_t)T * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        ctx->h2d += (size_t)T * sizeof(double);
        k_f64_to_f32<<<(T + 255) / 256, 256, 0, ctx->stream>>>(tmp, (size_t)T, o);
        count_launch();
        CU(cudaStreamSynchronize(ctx->stream));
        cudaFree(tmp);
    } else {
        double* o;
        CU(dalloc(&o, T));
        ctx->obs = o;
        CU(cudaMemcpyAsync(o, y, (size_t)T * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        ctx->h2d += (size_t)T * sizeof(double);
    }

    for (int b = 0; b < 2; ++b) {
        CU(dalloc(&ctx->theta[b], Ps * d));
        CU(dalloc(&ctx->ll[b], Ps));
        CU(dalloc(&ctx->lp[b], Ps));
        CU(dalloc(&ctx->state[b], Ps * (ctx->ns ? ctx->ns : 1)));
    }
    CU(dalloc(&ctx->thp, Ps * d));
    if (c->mutation == SMC_MALA) {
        CU(dalloc(&ctx->grad[0], Ps * d));
        CU(dalloc(&ctx->grad[1], Ps * d));
        CU(cudaMalloc(&ctx->ckpt, mala_ckpt_bytes(ctx->mdev, c->precision, T, P)));
    }
    CU(dalloc(&ctx->logw, Ps));
    CU(dalloc(&ctx->g, Ps * 3));
    CU(dalloc(&ctx->a, J));
    CU(dalloc(&ctx->a_score, J));
    if (c->pit) CU(dalloc(&ctx->pit, (size_t)T));
    CU(dalloc(&ctx->lw, J));
    CU(dalloc(&ctx->gstat, (size_t)J * 3));
    CU(dalloc(&ctx->idx, Ps));
    ctx->cov_G = cov_grid(P);
    CU(dalloc(&ctx->cov_part, (size_t)(ctx->cov_G + 1) * (d + d * (d + 1) / 2)));   // + totals row
    CU(dalloc(&ctx->search_part, search_part_len(P)));
    CU(cudaMemset(ctx->search_part, 0, search_bar_bytes()));
    CU(dalloc(&ctx->cd_part, cdata_part_len((P + kMutThreads - 1) / kMutThreads)));
    CU(cudaMemset(ctx->cd_part, 0, cdata_part_len((P + kMutThreads - 1) / kMutThreads) * sizeof(double)));
    if (c->tempering != SMC_POWER) CU(dalloc(&ctx->cd_end, Ps * (size_t)(1 + ctx->ns)));
    const int nf_max = d + 3;
    CU(dalloc(&ctx->mom_part, (size_t)nf_max * J * 2));
    CU(dalloc(&ctx->mom_out, (size_t)nf_max * 4));
    CU(dalloc(&ctx->ml_out, 3));
    CU(dalloc(&ctx->L, (size_t)d * d));
    CU(dalloc(&ctx->qmean, (size_t)d));
    {
        const int nacc = d + d * (d + 1) / 2;
        // the mutation kernels' compile-time parameter bound (Table 1 count)
        ctx->tile_kd = m->model == SMC_LINREG ? 8 : (m->I == 1 ? 2 + 3 * m->K : 2 + 3 * m->K + 3 * m->I);
        const int kd = ctx->tile_kd;
        ctx->ntiles = (P + 31) / 32;
        if (c->mutation != SMC_MALA) CU(dalloc(&ctx->covtile, (size_t)ctx->ntiles * (kd + kd * (kd + 1) / 2)));
        CU(dalloc(&ctx->covshift_f, (size_t)d));
        CU(dalloc(&ctx->cov_tot, (size_t)nacc));
        CU(dalloc(&ctx->cov_counter, 1));
        CU(cudaMemset(ctx->cov_counter, 0, sizeof(unsigned int)));
    }
    if (c->mutation == SMC_INDEP) CU(dalloc(&ctx->lq, Ps));
    CU(dalloc(&ctx->ctl, 1));
    CU(cudaMallocHost((void**)&ctx->ctl_host, 2 * sizeof(Ctl)));

    // gather tables: rows of theta, ll, lp, state for both directions
    const int ng = c->mutation == SMC_MALA ? d : 0;
    ctx->gather_rows = d + 2 + ctx->ns + ng;
    std::vector<double*> tab((size_t)2 * 2 * ctx->gather_rows);
    for (int dir = 0; dir < 2; ++dir) {
        const int from = dir, to = dir ^ 1;
        double** srcs = &tab[(size_t)dir * 2 * ctx->gather_rows];
        double** dsts = srcs + ctx->gather_rows;
        int r = 0;
        for (int i = 0; i < d; ++i, ++r) {
            srcs[r] = ctx->theta[from] + (size_t)i * Ps;
            dsts[r] = ctx->theta[to] + (size_t)i * Ps;
        }
        srcs[r] = ctx->ll[from];
        dsts[r++] = ctx->ll[to];
        srcs[r] = ctx->lp[from];
        dsts[r++] = ctx->lp[to];
        for (int k = 0; k < ctx->ns; ++k, ++r) {
            srcs[r] = ctx->state[from] + (size_t)k * Ps;
            dsts[r] = ctx->state[to] + (size_t)k * Ps;
        }
        for (int i = 0; i < ng; ++i, ++r) {
            srcs[r] = ctx->grad[from] + (size_t)i * Ps;
            dsts[r] = ctx->grad[to] + (size_t)i * Ps;
        }
    }
    CU(dalloc(&ctx->gather_ptrs, tab.size()));
    CU(cudaMemcpyAsync(ctx->gather_ptrs, tab.data(), tab.size() * sizeof(double*), cudaMemcpyHostToDevice,
                       ctx->stream));

    st = start_run(ctx, theta0, theta0_on_device);
    if (st != SMC_OK) return st;
    return SMC_OK;
}

}  // extern "C"

// Algorithm 1, step 1: particles from the prior, their log prior and (power
// tempering) full-sample log likelihood; estimator and control state zeroed.
static smc_status start_run(smc_ctx* ctx, const double* theta0, int theta0_on_device)
{
    const smc_config* c = &ctx->cfg;
    const int P = ctx->P, d = ctx->d, J = c->J, T = ctx->T;
    const size_t Ps = (size_t)P;
    if (theta0_on_device) {
        CU(cudaMemcpyAsync(ctx->theta[0], theta0, Ps * d * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
        CU(cudaMemcpyAsync(ctx->thp, theta0, Ps * d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        ctx->h2d += Ps * d * sizeof(double);
        const size_t n = Ps * d;
        k_to_soa<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->thp, P, d, ctx->theta[0]);
        count_launch();
    }
    Ctl init;
    std::memset(&init, 0, sizeof init);
    init.h_tenths = c->h0_tenths;
    CU(cudaMemcpyAsync(ctx->ctl, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->a, 0, (size_t)J * sizeof(double), ctx->stream));
    CU(cudaMemsetAsync(ctx->a_score, 0, (size_t)J * sizeof(double), ctx->stream));
    if (ctx->pit) CU(cudaMemsetAsync(ctx->pit, 0xff, (size_t)ctx->T * sizeof(double), ctx->stream));  // NaN
    if (c->tempering == SMC_POWER) {
        LoglikArgs la;
        la.m = ctx->mdev;
        la.obs = ctx->obs;
        la.T = T;
        la.W = ctx->W;
        la.theta = ctx->theta[0];
        la.ll = ctx->ll[0];
        la.lp = ctx->lp[0];
        la.state = ctx->ns ? ctx->state[0] : nullptr;
        la.P = P;
        la.ns = ctx->ns;
        la.err = &ctx->ctl->err;
        CU(launch_loglik(la, c->precision, ctx->stream));
        if (c->mutation == SMC_MALA) {
            smc_status st = refresh_gradient(ctx, T);
            if (st != SMC_OK) return st;
        }
    } else {
        k_init_data_tempering<<<(P + 255) / 256, 256, 0, ctx->stream>>>(ctx->mdev, ctx->theta[0], P,
                                                                        ctx->ns, ctx->ll[0], ctx->lp[0],
                                                                        ctx->state[0]);
        count_launch();
    }
    ctx->cur = 0;
    ctx->cycle = 0;
    ctx->t_prev = 0;
    ctx->done = 0;
    ctx->tiles_ready = false;   // the tile sums describe the previous particles
    ctx->phi = 0.0;
    ctx->msteps = 0;
    ctx->evals = 0.0;
    ctx->replay_iter = 0;
    if (ctx->record) {
        ctx->design_x.clear();
        ctx->design_R.clear();
        ctx->design_iters = 0;
    }
    return sync_ctl(ctx);
}

extern "C" {

smc_status smc_reset(smc_ctx* ctx, const double* theta0, int theta0_on_device, uint64_t seed)
{
    if (!ctx || !theta0) return SMC_EINVAL;
    ctx->cfg.seed = seed;
    return start_run(ctx, theta0, theta0_on_device);
}

smc_status smc_run_totals(smc_ctx* ctx, int* cycles, int64_t* metropolis_steps, double* evals)
{
    if (!ctx) return SMC_EINVAL;
    if (cycles) *cycles = ctx->cycle;
    if (metropolis_steps) *metropolis_steps = ctx->msteps;
    if (evals) *evals = ctx->evals;
    return SMC_OK;
}

smc_status smc_transfer_bytes(smc_ctx* ctx, uint64_t* h2d, uint64_t* d2h)
{
    if (!ctx) return SMC_EINVAL;
    if (h2d) *h2d = ctx->h2d;
    if (d2h) *d2h = ctx->d2h;
    return SMC_OK;
}

// Mutation launch-shape autotuner: times `iters` Metropolis iterations of each
// candidate shape on a snapshot of the particles (restored afterwards, with
// the control block) and keeps the fastest.
smc_status smc_autotune(smc_ctx* ctx, int iters, int* ppt, int* threads, double* ms_per_iteration)
{
    if (!ctx) return SMC_EINVAL;
    if (iters < 1) iters = 2;
    const bool fp32_egarch = ctx->model.model == SMC_EGARCH && ctx->cfg.precision == SMC_FP32 &&
                             ctx->cfg.mutation == SMC_RW;
    const int P = ctx->P, d = ctx->d;
    const size_t Ps = (size_t)P;
    const int from = ctx->cur, to = from ^ 1;
    CU(cudaMemcpyAsync(ctx->theta[to], ctx->theta[from], Ps * d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ll[to], ctx->ll[from], Ps * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->lp[to], ctx->lp[from], Ps * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->ns)
        CU(cudaMemcpyAsync(ctx->state[to], ctx->state[from], Ps * ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const Ctl saved = *ctx->ctl_host;
    struct Shape { int ppt, threads; };
    std::vector<Shape> cand = {{1, kMutThreads}};
    auto add = [&](int pp, int t) {
        for (const Shape& c : cand)
            if (c.ppt == pp && c.threads == t) return;
        cand.push_back({pp, t});
    };
    if (ctx->cfg.mutation != SMC_MALA) {
        add(1, 64);
        add(1, 32);
        add(1, balanced_threads(P, 1));
    }
    if (fp32_egarch) {
        add(2, 32);
        add(2, 64);
        add(2, 128);
        add(2, balanced_threads(P, 2));
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const int rec = ctx->record, prof = ctx->profile;
    ctx->record = 0;
    ctx->profile = 0;
    double best = 1e30;
    Shape pick = cand[0];
    const double phi = ctx->cfg.tempering == SMC_POWER ? ctx->phi : 1.0;
    const int Tm = ctx->cfg.tempering == SMC_POWER ? ctx->T : (ctx->t_prev > 0 ? ctx->t_prev : ctx->T);
    for (const Shape& sh : cand) {
        ctx->ppt = sh.ppt;
        ctx->mut_threads = sh.threads;
        smc_status st = m_iteration(ctx, 0, Tm, phi);   // warm-up
        if (st != SMC_OK) return st;
        CU(cudaEventRecord(e0, ctx->stream));
        for (int k = 0; k < iters; ++k) {
            st = m_iteration(ctx, k + 1, Tm, phi);
            if (st != SMC_OK) return st;
        }
        CU(cudaEventRecord(e1, ctx->stream));
        CU(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            pick = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->record = rec;
    ctx->profile = prof;
    ctx->ppt = pick.ppt;
    ctx->mut_threads = pick.threads;
    CU(cudaMemcpyAsync(ctx->theta[from], ctx->theta[to], Ps * d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ll[from], ctx->ll[to], Ps * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->lp[from], ctx->lp[to], Ps * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->ns)
        CU(cudaMemcpyAsync(ctx->state[from], ctx->state[to], Ps * ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    *ctx->ctl_host = saved;
    CU(cudaMemcpyAsync(ctx->ctl, ctx->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (ppt) *ppt = pick.ppt;
    if (threads) *threads = pick.threads;
    if (ms_per_iteration) *ms_per_iteration = best / iters;
    return SMC_OK;
}

smc_status smc_set_launch_shape(smc_ctx* ctx, int ppt, int threads)
{
    if (!ctx || ppt < 1 || ppt > 2 || !valid_mut_threads(threads)) return SMC_EINVAL;
    if (ppt == 2 && !(ctx->model.model == SMC_EGARCH && ctx->cfg.precision == SMC_FP32 &&
                      ctx->cfg.mutation == SMC_RW))
        return set_err(ctx, SMC_EINVAL, "two particles per thread needs the FP32 EGARCH random walk");
    ctx->ppt = ppt;
    ctx->mut_threads = threads;
    return SMC_OK;
}

smc_status smc_design_record(smc_ctx* ctx, int max_iterations)
{
    if (!ctx || max_iterations < 1) return SMC_EINVAL;
    if (ctx->replay) return set_err(ctx, SMC_EINVAL, "a replaying context cannot record");
    if (ctx->cfg.mutation == SMC_INDEP)
        return set_err(ctx, SMC_EINVAL, "a design holds no proposal means: the independent sampler cannot record");
    if (ctx->cycle > 0) return set_err(ctx, SMC_EINVAL, "start recording before the first cycle");
    if (ctx->design_L) cudaFree(ctx->design_L);
    ctx->design_L = nullptr;
    CU(cudaMalloc(&ctx->design_L, (size_t)max_iterations * ctx->d * ctx->d * sizeof(double)));
    ctx->design_cap = max_iterations;
    ctx->design_iters = 0;
    ctx->design_x.clear();
    ctx->design_R.clear();
    ctx->record = 1;
    return SMC_OK;
}

smc_status smc_design_size(smc_ctx* ctx, int* ncycles, int* niterations)
{
    if (!ctx) return SMC_EINVAL;
    if (ncycles) *ncycles = (int)ctx->design_x.size();
    if (niterations) *niterations = ctx->design_iters;
    return SMC_OK;
}

smc_status smc_design_get(smc_ctx* ctx, double* x, int* R, double* L)
{
    if (!ctx) return SMC_EINVAL;
    const int nc = (int)ctx->design_x.size();
    if (x) std::memcpy(x, ctx->design_x.data(), nc * sizeof(double));
    if (R) std::memcpy(R, ctx->design_R.data(), nc * sizeof(int));
    if (L && ctx->design_iters) {
        CU(cudaMemcpyAsync(L, ctx->design_L, (size_t)ctx->design_iters * ctx->d * ctx->d * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return SMC_OK;
}

smc_status smc_design_replay(smc_ctx* ctx, int ncycles, const double* x, const int* R, const double* L)
{
    if (!ctx || ncycles < 1 || !x || !R || !L) return SMC_EINVAL;
    if (ctx->cycle > 0) return set_err(ctx, SMC_EINVAL, "load the design before the first cycle");
    if (ctx->cfg.mutation != SMC_RW) return set_err(ctx, SMC_EINVAL, "replay takes random-walk runs");
    long iters = 0;
    for (int l = 0; l < ncycles; ++l) {
        if (R[l] < 0) return set_err(ctx, SMC_EINVAL, "negative iteration count");
        iters += R[l];
        if (ctx->cfg.tempering == SMC_DATA && (x[l] < 1 || x[l] > ctx->T || (l && x[l] <= x[l - 1])))
            return set_err(ctx, SMC_EINVAL, "data-tempering design must be increasing dates in 1..T");
        if (ctx->cfg.tempering == SMC_POWER && (!(x[l] > 0.0) || x[l] > 1.0 || (l && x[l] <= x[l - 1])))
            return set_err(ctx, SMC_EINVAL, "power design must be increasing powers in (0, 1]");
    }
    if (ctx->design_L) cudaFree(ctx->design_L);
    ctx->design_L = nullptr;
    const size_t bytes = (size_t)(iters > 0 ? iters : 1) * ctx->d * ctx->d * sizeof(double);
    CU(cudaMalloc(&ctx->design_L, bytes));
    if (iters) CU(cudaMemcpy(ctx->design_L, L, (size_t)iters * ctx->d * ctx->d * sizeof(double), cudaMemcpyHostToDevice));
    ctx->h2d += (uint64_t)iters * ctx->d * ctx->d * sizeof(double);
    ctx->design_x.assign(x, x + ncycles);
    ctx->design_R.assign(R, R + ncycles);
    ctx->design_iters = (int)iters;
    ctx->design_cap = (int)iters;
    ctx->replay_iter = 0;
    ctx->record = 0;
    ctx->replay = 1;
    return SMC_OK;
}

smc_status smc_profile(smc_ctx* ctx, int enable)
{
    if (!ctx) return SMC_EINVAL;
    if (enable < 0 || enable > 2) return set_err(ctx, SMC_EINVAL, "profile mode must be 0, 1 or 2");
    ctx->profile = enable;
    return SMC_OK;
}

smc_status smc_mutate_time(smc_ctx* ctx, double* ms, uint64_t* launches, int reset)
{
    if (!ctx) return SMC_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    smc_status st = fold_profile(ctx);
    if (st != SMC_OK) return st;
    if (ms) *ms = ctx->mutate_ms;
    if (launches) *launches = ctx->mutate_launches;
    if (reset) {
        ctx->mutate_ms = 0.0;
        ctx->mutate_launches = 0;
    }
    return SMC_OK;
}

// M phase of the current cycle (Algorithm 1, 2(c)): R Metropolis
// iterations, R from the stopping rule (the RNE rule reads the control block
// back after every iteration and may stop earlier), then the step-size update
// of the last iteration.  *ran = iterations run.  Enqueues only, apart from the
// RNE rule's read-backs.
static smc_status m_phase(smc_ctx* ctx, int Tm, double phim, double rss, int forced, int* ran)
{
    const smc_config& c = ctx->cfg;
    smc_status st;
    if (c.h_reset_each_cycle) {
        // the pending count (if any) was applied at the end of the last M phase
        int h0 = c.h0_tenths;
        CU(cudaMemcpyAsync(&ctx->ctl->h_tenths, &h0, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (c.mutation == SMC_MALA && c.tempering == SMC_DATA) {
        st = refresh_gradient(ctx, Tm);
        if (st != SMC_OK) return st;
    }
    const int R = ctx->replay ? ctx->design_R[ctx->cycle - 1] : smc_internal_R(ctx, rss);
    const double E = forced ? c.e2 : c.e1;
    int r = 0;
    for (; r < R; ++r) {
        st = m_iteration(ctx, r, Tm, phim);
        if (st != SMC_OK) return st;
        if (c.stop_rule == SMC_STOP_RNE) {
            st = test_functions(ctx, 1);
            if (st != SMC_OK) return st;
            st = sync_ctl(ctx);
            if (st != SMC_OK) return st;
            if (ctx->ctl_host->mean_rne >= E) {
                ++r;
                break;
            }
        }
    }
    *ran = r;
    return smc_internal_enqueue_adapt(ctx);
}

// One cycle's data-tempering C phase in progress (Algorithm 1, 2(a)):
// observations are absorbed in chunks of kCdataChunk until RSS < D1, a date
// of interest or T.  Chunks are queued in batches without waiting for the
// stop: each chunk's kernels do nothing once an earlier chunk of the cycle
// has found it (Ctl::cd_found), so a batch that overshoots costs only empty
// launches.  A cycle's first batch is as long as the previous cycle's C
// phase was; later batches take two chunks.
struct DataC {
    ForceDates fd;
    double d1 = 0.0;
    std::vector<int> start;   // start[seq]: observations absorbed before chunk seq (1-based)
    int s_next = 0;
    int batch = 1;
};

static smc_status data_c_enqueue(smc_ctx* ctx, DataC& dc)
{
    const smc_config& c = ctx->cfg;
    const int P = ctx->P;
    const int G = (P + kMutThreads - 1) / kMutThreads;
    for (int b = 0; b < dc.batch && dc.s_next < ctx->T; ++b) {
        const int seq = (int)dc.start.size();
        dc.start.push_back(dc.s_next);
        CdataArgs ca;
        ca.m = ctx->mdev;
        ca.obs = ctx->obs;
        ca.T = ctx->T;
        ca.W = ctx->W;
        ca.theta = ctx->theta[ctx->cur];
        ca.state = ctx->state[ctx->cur];
        ca.ll = ctx->ll[ctx->cur];
        ca.logw = ctx->logw;
        ca.P = P;
        ca.ns = ctx->ns;
        ca.s0 = dc.s_next;
        ca.B = ctx->T - dc.s_next < kCdataChunk ? ctx->T - dc.s_next : kCdataChunk;
        ca.part = ctx->cd_part;
        ca.end = ctx->cd_end;
        ca.stop = &ctx->ctl->cd_stop;
        ca.found = &ctx->ctl->cd_found;
        ca.seq = seq;
        ca.commit = 0;
        ca.pit = 0;
        ca.seed = c.seed;
        CU(launch_cdata(ca, c.precision, ctx->stream));
        CU(launch_cdata_select(ctx->cd_part, G, ca.B, dc.s_next, ctx->T, P, dc.d1, dc.fd, ctx->ctl, seq,
                               ctx->stream));
        ca.commit = 1;
        ca.pit = ctx->pit != nullptr;
        CU(launch_cdata(ca, c.precision, ctx->stream));
        if (ctx->pit) CU(launch_pit_final(ctx->cd_part, G, ca.B, dc.s_next, ctx->ctl, ctx->pit, seq, ctx->stream));
        dc.s_next += ca.B;
    }
    return SMC_OK;
}

// Enqueues the start of cycle `cycle`'s C phase from t_prev observations
// (weights reset, the first batch of chunks, the control block's read-back
// left to the caller).
static smc_status data_c_begin(smc_ctx* ctx, DataC& dc, int t_prev, int cycle)
{
    const smc_config& c = ctx->cfg;
    std::memset(&dc.fd, 0, sizeof dc.fd);
    dc.d1 = c.d1;
    if (ctx->replay) {
        if (cycle > (int)ctx->design_x.size())
            return set_err(ctx, SMC_EINVAL, "the replayed design has only %d cycles", (int)ctx->design_x.size());
        dc.fd.n = 1;
        dc.fd.t[0] = (int)ctx->design_x[cycle - 1];
        dc.d1 = -1.0;   // the recorded end, not RSS, closes the cycle
    } else {
        dc.fd.n = c.n_force;
        for (int i = 0; i < c.n_force; ++i) dc.fd.t[i] = c.force_dates[i];
        if (c.burnin > 0) dc.fd.t[dc.fd.n++] = c.burnin;   // the log score starts a cycle at b
    }
    dc.start.assign(1, 0);
    dc.s_next = t_prev;
    dc.batch = ctx->cd_chunks > 0 ? ctx->cd_chunks : 1;
    CU(cudaMemsetAsync(ctx->logw, 0, (size_t)ctx->P * sizeof(double), ctx->stream));
    CU(cudaMemsetAsync(&ctx->ctl->cd_found, 0, sizeof(int), ctx->stream));
    return data_c_enqueue(ctx, dc);
}

// With the control block of the latest batch read back: more batches until
// a chunk holds the stop, then the cycle's end t_l, its RSS and whether the
// end was forced.
static smc_status data_c_finish(smc_ctx* ctx, DataC& dc, int* t_l, double* rss, int* forced)
{
    for (;;) {
        const int f = ctx->ctl_host->cd_found;
        if (f > 0 && f < (int)dc.start.size()) {
            *t_l = dc.start[f] + ctx->ctl_host->cd_stop;
            *rss = ctx->ctl_host->rss;
            *forced = ctx->ctl_host->cd_forced || *t_l == ctx->T;
            ctx->cd_chunks = f;
            return SMC_OK;
        }
        if (f != 0 || dc.s_next >= ctx->T)
            return set_err(ctx, SMC_ECUDA, "data tempering: no stop found by observation %d", dc.s_next);
        dc.batch = 2;
        smc_status st = data_c_enqueue(ctx, dc);
        if (st != SMC_OK) return st;
        st = sync_ctl(ctx);
        if (st != SMC_OK) return st;
    }
}

smc_status smc_cycle(smc_ctx* ctx, smc_cycle_info* info)
{
    if (!ctx) return SMC_EINVAL;
    if (ctx->done) return set_err(ctx, SMC_EDONE, "the run has reached the full posterior");
    const smc_config& c = ctx->cfg;
    if (c.tempering != SMC_POWER) ctx->cycle += 1;
    int t_l = ctx->T;
    double rss = 1.0;
    int forced = 0;
    smc_status st;
    if (c.tempering == SMC_POWER) {
        st = smc_internal_enqueue_cs(ctx);
        if (st != SMC_OK) return st;
        st = sync_ctl(ctx);
        if (st != SMC_OK) return st;
        smc_internal_after_cs(ctx, &rss, &forced);
    } else {
        // ---- C phase: add observations until RSS < D1 (Algorithm 1, 2(a)) ----
        DataC dc;
        st = data_c_begin(ctx, dc, ctx->t_prev, ctx->cycle);
        if (st != SMC_OK) return st;
        st = sync_ctl(ctx);
        if (st != SMC_OK) return st;
        st = data_c_finish(ctx, dc, &t_l, &rss, &forced);
        if (st != SMC_OK) return st;
        // ---- S phase (weights from the accumulated log weights) ----
        st = s_phase(ctx, 1);
        if (st != SMC_OK) return st;
        CU(launch_cycle_close(ctx->gstat, ctx->lw, c.J, c.N, 0, ctx->ctl, ctx->stream));
        ctx->phi = 1.0;
    }
    // ---- M phase ----
    const double phim = c.tempering == SMC_POWER ? ctx->phi : 1.0;
    const int Tm = c.tempering == SMC_POWER ? ctx->T : t_l;
    int r = 0;
    st = m_phase(ctx, Tm, phim, rss, forced, &r);
    if (st != SMC_OK) return st;
    st = sync_ctl(ctx);
    if (st != SMC_OK) return st;
    return smc_internal_after_m(ctx, t_l, r, Tm, phim, rss, info);
}

// Power tempering, cycle after cycle with one host round trip per cycle:
// while the run goes on, the next cycle's C and S phases are enqueued right
// behind this cycle's M phase, and one synchronisation returns both the
// M phase's control block (ctl_host[1]) and the next C phase's (ctl_host[0]).
// The kernels and their order are those of smc_cycle; only the host waits
// differently.
static smc_status run_power_pipelined(smc_ctx* ctx, int max_cycles, smc_cycle_info* info, int* ncycles)
{
    int n = 0;
    smc_cycle_info ci;
    std::memset(&ci, 0, sizeof ci);
    Ctl* hm = ctx->ctl_host + 1;
    bool have_cs = false;   // this cycle's C and S phases are enqueued and read back
    double rss = 1.0;
    int forced = 0;
    smc_status st = SMC_OK;
    while (!ctx->done && (max_cycles <= 0 || n < max_cycles)) {
        if (!have_cs) {
            st = smc_internal_enqueue_cs(ctx);
            if (st != SMC_OK) break;
            st = sync_ctl(ctx);
            if (st != SMC_OK) break;
            smc_internal_after_cs(ctx, &rss, &forced);
        }
        const int cycle = ctx->cycle;
        const double phim = ctx->phi;
        int r = 0;
        st = m_phase(ctx, ctx->T, phim, rss, forced, &r);
        if (st != SMC_OK) break;
        CU(cudaMemcpyAsync(hm, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
        ctx->d2h += sizeof(Ctl);
        // forced = this C phase took the remaining power (the last cycle)
        have_cs = !forced && (max_cycles <= 0 || n + 1 < max_cycles);
        if (have_cs) {
            st = smc_internal_enqueue_cs(ctx);
            if (st != SMC_OK) break;
            st = smc_internal_enqueue_ctl_readback(ctx);
            if (st != SMC_OK) break;
        }
        CU(cudaStreamSynchronize(ctx->stream));
        // the error word is sticky: the later read-back carries every error
        st = check_device_error(ctx, have_cs ? *ctx->ctl_host : *hm);
        if (st != SMC_OK) break;
        st = after_m_from(ctx, *hm, cycle, ctx->T, r, ctx->T, phim, rss, &ci);
        if (st != SMC_OK) break;
        ++n;
        if (have_cs) smc_internal_after_cs(ctx, &rss, &forced);
    }
    if (info) *info = ci;
    if (ncycles) *ncycles = n;
    return st;
}

// Data tempering, likewise: the next cycle's C phase starts (its first batch
// of chunks) right behind this cycle's M phase, and one synchronisation
// returns the M phase's control block (ctl_host[1]) and the batch's
// (ctl_host[0]).  The kernels and their order are those of smc_cycle.
static smc_status run_data_pipelined(smc_ctx* ctx, int max_cycles, smc_cycle_info* info, int* ncycles)
{
    const smc_config& c = ctx->cfg;
    int n = 0;
    smc_cycle_info ci;
    std::memset(&ci, 0, sizeof ci);
    Ctl* hm = ctx->ctl_host + 1;
    bool have_c = false;   // this cycle's first batch is enqueued and read back
    DataC dc;
    smc_status st = SMC_OK;
    while (!ctx->done && (max_cycles <= 0 || n < max_cycles)) {
        if (!have_c) {
            ctx->cycle += 1;
            st = data_c_begin(ctx, dc, ctx->t_prev, ctx->cycle);
            if (st != SMC_OK) break;
            st = sync_ctl(ctx);
            if (st != SMC_OK) break;
        }
        int t_l = ctx->T, forced = 0;
        double rss = 1.0;
        st = data_c_finish(ctx, dc, &t_l, &rss, &forced);
        if (st != SMC_OK) break;
        st = s_phase(ctx, 1);
        if (st != SMC_OK) break;
        CU(launch_cycle_close(ctx->gstat, ctx->lw, c.J, c.N, 0, ctx->ctl, ctx->stream));
        ctx->phi = 1.0;
        const int cycle = ctx->cycle;
        int r = 0;
        st = m_phase(ctx, t_l, 1.0, rss, forced, &r);
        if (st != SMC_OK) break;
        CU(cudaMemcpyAsync(hm, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
        ctx->d2h += sizeof(Ctl);
        have_c = t_l < ctx->T && (max_cycles <= 0 || n + 1 < max_cycles) &&
                 (!ctx->replay || cycle < (int)ctx->design_x.size());
        if (have_c) {
            ctx->cycle += 1;
            st = data_c_begin(ctx, dc, t_l, ctx->cycle);
            if (st != SMC_OK) break;
            st = smc_internal_enqueue_ctl_readback(ctx);
            if (st != SMC_OK) break;
        }
        CU(cudaStreamSynchronize(ctx->stream));
        // the error word is sticky: the later read-back carries every error
        st = check_device_error(ctx, have_c ? *ctx->ctl_host : *hm);
        if (st != SMC_OK) break;
        st = after_m_from(ctx, *hm, cycle, t_l, r, t_l, 1.0, rss, &ci);
        if (st != SMC_OK) break;
        ++n;
    }
    if (info) *info = ci;
    if (ncycles) *ncycles = n;
    return st;
}

smc_status smc_run(smc_ctx* ctx, int max_cycles, smc_cycle_info* info, int* ncycles)
{
    if (!ctx) return SMC_EINVAL;
    if (ctx->cfg.tempering == SMC_POWER && !ctx->done) return run_power_pipelined(ctx, max_cycles, info, ncycles);
    if (ctx->cfg.tempering == SMC_DATA && !ctx->done) return run_data_pipelined(ctx, max_cycles, info, ncycles);
    int n = 0;
    smc_cycle_info ci;
    std::memset(&ci, 0, sizeof ci);
    while (!ctx->done && (max_cycles <= 0 || n < max_cycles)) {
        smc_status st = smc_cycle(ctx, &ci);
        if (st != SMC_OK) {
            if (ncycles) *ncycles = n;
            return st;
        }
        ++n;
    }
    if (info) *info = ci;
    if (ncycles) *ncycles = n;
    return SMC_OK;
}

smc_status smc_log_ml(smc_ctx* ctx, double* log_ml, double* nse, double* log_ml_tilde)
{
    if (!ctx) return SMC_EINVAL;
    CU(launch_ml(ctx->a, ctx->cfg.J, ctx->ctl, ctx->ml_out, ctx->stream));
    double h[3];
    CU(cudaMemcpyAsync(h, ctx->ml_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->d2h += sizeof h;
    CU(cudaStreamSynchronize(ctx->stream));
    if (log_ml) *log_ml = h[0];
    if (nse) *nse = h[1];
    if (log_ml_tilde) *log_ml_tilde = h[2];
    return SMC_OK;
}

smc_status smc_group_estimators(smc_ctx* ctx, double* a, double* lw)
{
    if (!ctx) return SMC_EINVAL;
    const size_t bytes = (size_t)ctx->cfg.J * sizeof(double);
    if (a) {
        CU(cudaMemcpyAsync(a, ctx->a, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        ctx->d2h += bytes;
    }
    if (lw) {
        CU(cudaMemcpyAsync(lw, ctx->lw, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        ctx->d2h += bytes;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return SMC_OK;
}

smc_status smc_moments(smc_ctx* ctx, double* out, int* nf)
{
    if (!ctx || !out) return SMC_EINVAL;
    const int d = ctx->d, J = ctx->cfg.J, N = ctx->cfg.N;
    CU(launch_moments(ctx->theta[ctx->cur], d, J, N, ctx->mom_part, ctx->mom_out, nullptr, 0, ctx->stream));
    CU(cudaMemcpyAsync(out, ctx->mom_out, (size_t)d * 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    int n = d;
    if (ctx->model.model == SMC_EGARCH) {
        CU(launch_testfn(ctx->mdev, ctx->cfg.precision, ctx->theta[ctx->cur], ctx->state[ctx->cur], ctx->P,
                         ctx->g, ctx->stream));
        CU(launch_moments(ctx->g, 3, J, N, ctx->mom_part, ctx->mom_out, nullptr, 0, ctx->stream));
        CU(cudaMemcpyAsync(out + (size_t)d * 4, ctx->mom_out, 3 * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
        n += 3;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    if (nf) *nf = n;
    return SMC_OK;
}

smc_status smc_get_particles(smc_ctx* ctx, double* theta, double* loglik, double* logprior, double* state)
{
    if (!ctx) return SMC_EINVAL;
    const int P = ctx->P, d = ctx->d;
    const size_t Ps = (size_t)P;
    if (theta) {
        const size_t n = Ps * d;
        k_to_aos<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->theta[ctx->cur], P, d, ctx->thp);
        count_launch();
        CU(cudaMemcpyAsync(theta, ctx->thp, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (loglik) CU(cudaMemcpyAsync(loglik, ctx->ll[ctx->cur], Ps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (logprior) CU(cudaMemcpyAsync(logprior, ctx->lp[ctx->cur], Ps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (state && ctx->ns) {
        CU(cudaStreamSynchronize(ctx->stream));
        const size_t n = Ps * ctx->ns;
        k_to_aos<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->state[ctx->cur], P, ctx->ns, ctx->thp);
        count_launch();
        CU(cudaMemcpyAsync(state, ctx->thp, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return SMC_OK;
}

smc_status smc_log_score(smc_ctx* ctx, double* log_score, double* nse)
{
    if (!ctx || !log_score) return SMC_EINVAL;
    if (ctx->cfg.burnin <= 0) return set_err(ctx, SMC_EINVAL, "no burn-in was set");
    CU(launch_ml(ctx->a_score, ctx->cfg.J, ctx->ctl, ctx->ml_out, ctx->stream));
    double out[3];
    CU(cudaMemcpyAsync(out, ctx->ml_out, sizeof out, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *log_score = out[0];
    if (nse) *nse = out[1];
    return SMC_OK;
}

smc_status smc_pit(smc_ctx* ctx, double* out, int T)
{
    if (!ctx || !out || T != ctx->T) return SMC_EINVAL;
    if (!ctx->pit) return set_err(ctx, SMC_EINVAL, "the context was created without pit = 1");
    CU(cudaMemcpyAsync(out, ctx->pit, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return SMC_OK;
}

void smc_free(smc_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    release(ctx);
    delete ctx;
}

}  // extern "C"
