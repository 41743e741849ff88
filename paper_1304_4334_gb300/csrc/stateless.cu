// Stateless entry points of the C ABI: each phase kernel on caller-owned device
// memory, for tests, the autograd binding and custom drivers.  Temporaries are
// allocated stream-ordered on the caller's stream and freed before returning.
#include "../../include/smc.h"
#include "kernels.cuh"
#include "mala.cuh"
#include "phase.cuh"

#include <cmath>
#include <cstring>

namespace smc {
void count_launch();
}
using namespace smc;

namespace {

void model_dev(const smc_model& m, ModelDev& d)
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

bool model_ok(const smc_model* m, int precision)
{
    if (!m) return false;
    if (m->model == SMC_EGARCH) {
        if (m->K < 1 || m->K > kMaxK || m->I < 1 || m->I > kMaxI) return false;
        if (precision != SMC_FP32 && precision != SMC_FP64) return false;
    } else if (m->model == SMC_LINREG) {
        if (m->p < 1 || m->p > 7 || precision != SMC_FP64) return false;
    } else {
        return false;
    }
    return m->d_full >= 1 && m->d_full <= SMC_MAX_D && m->n_free >= 0 && m->n_free <= m->d_full;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

smc_status from_cuda(cudaError_t e) { return e == cudaSuccess ? SMC_OK : SMC_ECUDA; }

}  // namespace

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return SMC_ECUDA; \
    } while (0)

extern "C" {

smc_status smc_loglik(const smc_model* m, int precision, const void* obs, int T, const double* theta,
                      int P, double* ll, double* lp, double* state, void* stream)
{
    if (!model_ok(m, precision) || !obs || !theta || !ll || T < 1 || P < 1 || !aligned16(obs))
        return SMC_EINVAL;
    LoglikArgs a;
    a.m = ModelDev{};
    model_dev(*m, a.m);
    a.obs = obs;
    a.T = T;
    a.W = m->model == SMC_LINREG ? smc_linreg_width(m->p) : 1;
    a.theta = theta;
    a.ll = ll;
    a.lp = lp;
    a.state = m->model == SMC_EGARCH ? state : nullptr;
    a.P = P;
    a.ns = m->model == SMC_EGARCH ? m->K + 1 : 0;
    a.err = nullptr;
    return from_cuda(launch_loglik(a, precision, (cudaStream_t)stream));
}

static smc_status mutate_impl(const smc_model* m, int precision, const void* obs, int T, double* theta,
                              double* ll, double* lp, double* state, int P, const double* qmean,
                              const double* L, double phi, uint64_t seed, uint64_t cycle, uint64_t iter,
                              uint64_t* accepted, void* stream)
{
    if (!model_ok(m, precision) || !obs || !theta || !ll || !lp || !L || T < 1 || P < 1 ||
        !aligned16(obs) || !(phi >= 0.0))
        return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int d = m->n_free > 0 ? m->n_free : m->d_full;
    double* thp = nullptr;
    unsigned long long* cnt = nullptr;
    CK(cudaMallocAsync((void**)&thp, (size_t)P * d * sizeof(double), s));
    CK(cudaMallocAsync((void**)&cnt, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    double* lq = nullptr;
    if (qmean) {
        CK(cudaMallocAsync((void**)&lq, (size_t)P * sizeof(double), s));
        CK(launch_indep_logq(theta, d, P, L, qmean, lq, s));
    }
    MutateArgs a;
    a.m = ModelDev{};
    model_dev(*m, a.m);
    a.obs = obs;
    a.T = T;
    a.W = m->model == SMC_LINREG ? smc_linreg_width(m->p) : 1;
    a.theta = theta;
    a.ll = ll;
    a.lp = lp;
    a.state = m->model == SMC_EGARCH ? state : nullptr;
    a.thp = thp;
    a.P = P;
    a.ns = m->model == SMC_EGARCH ? m->K + 1 : 0;
    a.L = L;
    a.qmean = qmean;
    a.lq = lq;
    a.covtile = nullptr;
    a.covshift = nullptr;
    a.ntiles = 0;
    a.phi = phi;
    a.seed = seed;
    a.cycle = cycle;
    a.iter = iter;
    a.acc_count = cnt;
    a.pending = nullptr;
    a.err = nullptr;
    cudaError_t e = launch_mutate(a, precision, kMutThreads, s);
    unsigned long long h = 0;
    if (e == cudaSuccess && accepted) {
        e = cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *accepted = h;
    }
    cudaFreeAsync(thp, s);
    cudaFreeAsync(cnt, s);
    if (lq) cudaFreeAsync(lq, s);
    return from_cuda(e);
}

smc_status smc_mutate_rw(const smc_model* m, int precision, const void* obs, int T, double* theta,
                         double* ll, double* lp, double* state, int P, const double* L, double phi,
                         uint64_t seed, uint64_t cycle, uint64_t iter, uint64_t* accepted,
                         void* stream)
{
    return mutate_impl(m, precision, obs, T, theta, ll, lp, state, P, nullptr, L, phi, seed, cycle,
                       iter, accepted, stream);
}

smc_status smc_mutate_indep(const smc_model* m, int precision, const void* obs, int T, double* theta,
                            double* ll, double* lp, double* state, int P, const double* mean,
                            const double* L, double phi, uint64_t seed, uint64_t cycle, uint64_t iter,
                            uint64_t* accepted, void* stream)
{
    if (!mean) return SMC_EINVAL;
    return mutate_impl(m, precision, obs, T, theta, ll, lp, state, P, mean, L, phi, seed, cycle,
                       iter, accepted, stream);
}

smc_status smc_loglik_grad(const smc_model* m, int precision, const void* obs, int T,
                           const double* theta, int P, double* ll, double* grad, double* state,
                           void* stream)
{
    if (!model_ok(m, precision) || !obs || !theta || !ll || !grad || T < 1 || P < 1 || !aligned16(obs))
        return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    GradArgs a;
    a.m = ModelDev{};
    model_dev(*m, a.m);
    a.obs = obs;
    a.T = T;
    a.W = m->model == SMC_LINREG ? smc_linreg_width(m->p) : 1;
    a.theta = theta;
    a.P = P;
    a.ll = ll;
    a.grad = grad;
    a.state = m->model == SMC_EGARCH ? state : nullptr;
    a.ckpt = nullptr;
    CK(cudaMallocAsync(&a.ckpt, mala_ckpt_bytes(a.m, precision, T, P), s));
    const cudaError_t e = launch_loglik_grad(a, precision, s);
    cudaFreeAsync(a.ckpt, s);
    return from_cuda(e);
}

smc_status smc_mutate_mala(const smc_model* m, int precision, const void* obs, int T, double* theta,
                           double* ll, double* lp, double* grad, double* state, int P, const double* L,
                           double phi, uint64_t seed, uint64_t cycle, uint64_t iter, uint64_t* accepted,
                           void* stream)
{
    if (!model_ok(m, precision) || !obs || !theta || !ll || !lp || !grad || !L || T < 1 || P < 1 ||
        !aligned16(obs) || !(phi >= 0.0))
        return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* cnt = nullptr;
    MalaArgs a;
    a.m = ModelDev{};
    model_dev(*m, a.m);
    a.obs = obs;
    a.T = T;
    a.W = m->model == SMC_LINREG ? smc_linreg_width(m->p) : 1;
    a.theta = theta;
    a.ll = ll;
    a.lp = lp;
    a.state = m->model == SMC_EGARCH ? state : nullptr;
    a.grad = grad;
    a.ckpt = nullptr;
    a.P = P;
    a.ns = m->model == SMC_EGARCH ? m->K + 1 : 0;
    a.L = L;
    a.phi = phi;
    a.seed = seed;
    a.cycle = cycle;
    a.iter = iter;
    a.pending = nullptr;
    a.err = nullptr;
    CK(cudaMallocAsync(&a.ckpt, mala_ckpt_bytes(a.m, precision, T, P), s));
    CK(cudaMallocAsync((void**)&cnt, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    a.acc_count = cnt;
    cudaError_t e = launch_mala(a, precision, s);
    unsigned long long h = 0;
    if (e == cudaSuccess && accepted) {
        e = cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *accepted = h;
    }
    cudaFreeAsync(a.ckpt, s);
    cudaFreeAsync(cnt, s);
    return from_cuda(e);
}

smc_status smc_cov_chol(const double* theta, int d, int P, int h_tenths, double* mean, double* cov,
                        double* L, void* stream)
{
    if (!theta || d < 1 || d > SMC_MAX_D || P < 2 || h_tenths < 0) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = cov_grid(P);
    double* part = nullptr;
    const size_t n = (size_t)(G + 1) * (d + d * (d + 1) / 2);
    CK(cudaMallocAsync((void**)&part, (n + 1) * sizeof(double), s));
    unsigned int* counter = reinterpret_cast<unsigned int*>(part + n);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
    cudaError_t e = launch_cov(theta, d, P, part, G, counter, nullptr, h_tenths, 0.0, 1, 10, mean, cov, L, s);
    cudaFreeAsync(part, s);
    return from_cuda(e);
}

smc_status smc_power_search(const double* ll, int P, double phi, double d1, int passes, double* dphi,
                            double* rss, void* stream)
{
    if (!ll || P < 1 || !(phi >= 0.0 && phi < 1.0) || !(d1 > 0.0 && d1 < 1.0) || passes < 1)
        return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double* part = nullptr;
    Ctl* ctl = nullptr;
    double* gstat = nullptr;
    double* lw = nullptr;
    double* a = nullptr;
    int32_t* idx = nullptr;
    CK(cudaMallocAsync((void**)&part, search_part_len(P) * sizeof(double), s));
    CK(cudaMemsetAsync(part, 0, search_bar_bytes(), s));
    CK(cudaMallocAsync((void**)&ctl, sizeof(Ctl), s));
    CK(cudaMallocAsync((void**)&gstat, 3 * sizeof(double), s));
    CK(cudaMallocAsync((void**)&lw, sizeof(double), s));
    CK(cudaMallocAsync((void**)&a, sizeof(double), s));
    CK(cudaMallocAsync((void**)&idx, (size_t)P * sizeof(int32_t), s));
    Ctl init;
    std::memset(&init, 0, sizeof init);
    init.phi = phi;
    cudaError_t e = cudaMemcpyAsync(ctl, &init, sizeof init, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_power_search(ll, P, d1, passes, part, ctl, s);
    // FP64 RSS at the chosen power: the weights pass of the S phase over one
    // group holding all particles gives (max, sum w, sum w^2).
    if (e == cudaSuccess && P <= SMC_MAX_N) {
        SelectArgs sa;
        std::memset(&sa, 0, sizeof sa);
        sa.mode = 0;
        sa.ll = ll;
        sa.J = 1;
        sa.N = P;
        sa.scheme = 0;
        sa.a = a;
        sa.lw = lw;
        sa.gstat = gstat;
        sa.idx = idx;
        sa.ctl = ctl;
        CK(cudaMemsetAsync(a, 0, sizeof(double), s));
        e = launch_select(sa, s);
        if (e == cudaSuccess) e = launch_cycle_close(gstat, lw, 1, P, 0, ctl, s);
    }
    Ctl h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        if (dphi) *dphi = h.dphi;
        if (rss) *rss = P <= SMC_MAX_N ? h.rss : NAN;
    }
    cudaFreeAsync(part, s);
    cudaFreeAsync(ctl, s);
    cudaFreeAsync(gstat, s);
    cudaFreeAsync(lw, s);
    cudaFreeAsync(a, s);
    cudaFreeAsync(idx, s);
    return from_cuda(e);
}

smc_status smc_resample(const double* w, int J, int N, int resampler, uint64_t seed, uint64_t cycle,
                        int32_t* idx, void* stream)
{
    if (!w || !idx || J < 1 || N < 1 || N > SMC_MAX_N) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int* err = nullptr;
    CK(cudaMallocAsync((void**)&err, sizeof(int), s));
    CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    SelectArgs sa;
    std::memset(&sa, 0, sizeof sa);
    sa.mode = 2;
    sa.w = w;
    sa.J = J;
    sa.N = N;
    sa.scheme = resampler;
    sa.seed = seed;
    sa.cycle = cycle;
    sa.idx = idx;
    sa.err = err;
    cudaError_t e = launch_select(sa, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(err, s);
    if (e != cudaSuccess) return SMC_ECUDA;
    if (h & kErrDegenerate) return SMC_EDEGENERATE;
    return h ? SMC_ECUDA : SMC_OK;
}

smc_status smc_resample_logw(const double* logw, int J, int N, int resampler, uint64_t seed, uint64_t cycle,
                             int32_t* idx, double* lwbar, void* stream)
{
    if (!logw || !idx || J < 1 || N < 1 || N > SMC_MAX_N || resampler < 0 || resampler > 3) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int* err = nullptr;
    double* buf = nullptr;   // a [J], lw [J], gstat [3 J]
    CK(cudaMallocAsync((void**)&err, sizeof(int), s));
    CK(cudaMallocAsync((void**)&buf, (size_t)5 * J * sizeof(double), s));
    CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    CK(cudaMemsetAsync(buf, 0, (size_t)J * sizeof(double), s));
    SelectArgs sa;
    std::memset(&sa, 0, sizeof sa);
    sa.mode = 1;
    sa.logw = logw;
    sa.J = J;
    sa.N = N;
    sa.scheme = resampler;
    sa.seed = seed;
    sa.cycle = cycle;
    sa.a = buf;
    sa.lw = buf + J;
    sa.gstat = buf + 2 * J;
    sa.idx = idx;
    sa.err = err;
    cudaError_t e = launch_select(sa, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && lwbar)
        e = cudaMemcpyAsync(lwbar, buf + J, (size_t)J * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(err, s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return SMC_ECUDA;
    if (h & kErrDegenerate) return SMC_EDEGENERATE;
    return h ? SMC_ECUDA : SMC_OK;
}

smc_status smc_group_moments(const double* g, int nf, int J, int N, double* out, void* stream)
{
    if (!g || !out || nf < 1 || J < 2 || N < 1) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double* part = nullptr;
    double* dout = nullptr;
    CK(cudaMallocAsync((void**)&part, (size_t)nf * J * 2 * sizeof(double), s));
    CK(cudaMallocAsync((void**)&dout, (size_t)nf * 4 * sizeof(double), s));
    cudaError_t e = launch_moments(g, nf, J, N, part, dout, nullptr, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)nf * 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(dout, s);
    return from_cuda(e);
}

smc_status smc_ml_from_groups(const double* a, int J, double* log_ml, double* nse, void* stream)
{
    if (!a || J < 2) return SMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double* dout = nullptr;
    CK(cudaMallocAsync((void**)&dout, 3 * sizeof(double), s));
    cudaError_t e = launch_ml(a, J, nullptr, dout, s);
    double h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(dout, s);
    if (log_ml) *log_ml = h[0];
    if (nse) *nse = h[1];
    return from_cuda(e);
}

}  // extern "C"
