// Checkpoint and resume of a simulator context between cycles.
//
// A run is a deterministic function of its inputs and of the Philox counters
// (particle, iteration, cycle, tag), so saving the state that survives a cycle
// boundary and restoring it into a fresh context continues the run exactly:
// the model, the settings, the observations, the current particles (theta, log
// likelihood, log prior, recursion state, MALA gradient), the per-group
// log-ML and log-score accumulators, the PIT values, the device control block
// (step size, power, log wtilde, acceptance bookkeeping), the host run state
// and the hybrid design being recorded or replayed.  Everything else a cycle
// uses (weights, covariance, partial sums) is recomputed inside the cycle.
#include "ctx.h"

#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

namespace {

constexpr char kMagic[8] = {'S', 'M', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

struct Header {
    char magic[8];
    uint32_t version, sz_model, sz_config, sz_ctl;
    int32_t T, P, d, ns, W, mala, has_pit;
    int32_t cycle, t_prev, done, record, replay, design_iters, design_cap, replay_iter, ndesign;
    int32_t ppt, mut_threads;
    double phi, evals;
    int64_t msteps;
};

struct File {
    FILE* f = nullptr;
    ~File()
    {
        if (f) fclose(f);
    }
};

bool put(FILE* f, const void* p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }

template <typename T>
cudaError_t d2h(std::vector<T>& v, const void* src, size_t n)
{
    v.resize(n);
    return n ? cudaMemcpy(v.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) : cudaSuccess;
}

template <typename T>
bool put_vec(FILE* f, const std::vector<T>& v)
{
    return put(f, v.data(), v.size() * sizeof(T));
}

}  // namespace

extern "C" smc_status smc_save(smc_ctx* ctx, const char* path)
{
    if (!ctx || !path) return SMC_EINVAL;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return SMC_ECUDA;
    const size_t P = (size_t)ctx->P, d = (size_t)ctx->d, ns = (size_t)ctx->ns, T = (size_t)ctx->T;
    const size_t J = (size_t)ctx->cfg.J;
    const bool mala = ctx->cfg.mutation == SMC_MALA;
    const bool f32obs = ctx->model.model == SMC_EGARCH && ctx->cfg.precision == SMC_FP32;
    Header h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = kVersion;
    h.sz_model = sizeof(smc_model);
    h.sz_config = sizeof(smc_config);
    h.sz_ctl = sizeof(Ctl);
    h.T = ctx->T;
    h.P = ctx->P;
    h.d = ctx->d;
    h.ns = ctx->ns;
    h.W = ctx->W;
    h.mala = mala;
    h.has_pit = ctx->pit != nullptr;
    h.cycle = ctx->cycle;
    h.t_prev = ctx->t_prev;
    h.done = ctx->done;
    h.record = ctx->record;
    h.replay = ctx->replay;
    h.design_iters = ctx->design_iters;
    h.design_cap = ctx->design_cap;
    h.replay_iter = ctx->replay_iter;
    h.ndesign = (int32_t)ctx->design_x.size();
    h.ppt = ctx->ppt;
    h.mut_threads = ctx->mut_threads;
    h.phi = ctx->phi;
    h.evals = ctx->evals;
    h.msteps = ctx->msteps;

    std::vector<float> obs_f;
    std::vector<double> obs_d, th, ll, lp, st, gr, a, as, pit, dl;
    cudaError_t e = cudaSuccess;
    if (f32obs) e = d2h(obs_f, ctx->obs, T);
    else e = d2h(obs_d, ctx->obs, T * (size_t)ctx->W);
    const int c = ctx->cur;
    if (e == cudaSuccess) e = d2h(th, ctx->theta[c], d * P);
    if (e == cudaSuccess) e = d2h(ll, ctx->ll[c], P);
    if (e == cudaSuccess) e = d2h(lp, ctx->lp[c], P);
    if (e == cudaSuccess && ns) e = d2h(st, ctx->state[c], ns * P);
    if (e == cudaSuccess && mala) e = d2h(gr, ctx->grad[c], d * P);
    if (e == cudaSuccess) e = d2h(a, ctx->a, J);
    if (e == cudaSuccess) e = d2h(as, ctx->a_score, J);
    if (e == cudaSuccess && ctx->pit) e = d2h(pit, ctx->pit, T);
    if (e == cudaSuccess && ctx->design_L && ctx->design_iters)
        e = d2h(dl, ctx->design_L, (size_t)ctx->design_iters * d * d);
    Ctl ctl;
    if (e == cudaSuccess) e = cudaMemcpy(&ctl, ctx->ctl, sizeof ctl, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return SMC_ECUDA;

    File out;
    out.f = std::fopen(path, "wb");
    if (!out.f) {
        ctx->err = "cannot open the checkpoint file for writing";
        return SMC_EINVAL;
    }
    bool ok = put(out.f, &h, sizeof h) && put(out.f, &ctx->model, sizeof ctx->model) &&
              put(out.f, &ctx->cfg, sizeof ctx->cfg) && put(out.f, &ctl, sizeof ctl) &&
              put_vec(out.f, obs_f) && put_vec(out.f, obs_d) && put_vec(out.f, th) && put_vec(out.f, ll) &&
              put_vec(out.f, lp) && put_vec(out.f, st) && put_vec(out.f, gr) && put_vec(out.f, a) &&
              put_vec(out.f, as) && put_vec(out.f, pit) && put_vec(out.f, ctx->design_x) &&
              put_vec(out.f, ctx->design_R) && put_vec(out.f, dl);
    ok = ok && std::fflush(out.f) == 0;
    if (!ok) {
        ctx->err = "writing the checkpoint file failed";
        return SMC_EINVAL;
    }
    return SMC_OK;
}

extern "C" smc_status smc_load(const char* path, void* stream, smc_ctx** out)
{
    if (!path || !out) return SMC_EINVAL;
    *out = nullptr;
    File in;
    in.f = std::fopen(path, "rb");
    if (!in.f) return SMC_EINVAL;
    Header h;
    smc_model m;
    smc_config c;
    Ctl ctl;
    if (!get(in.f, &h, sizeof h) || std::memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.version != kVersion ||
        h.sz_model != sizeof(smc_model) || h.sz_config != sizeof(smc_config) || h.sz_ctl != sizeof(Ctl))
        return SMC_EINVAL;
    if (!get(in.f, &m, sizeof m) || !get(in.f, &c, sizeof c) || !get(in.f, &ctl, sizeof ctl)) return SMC_EINVAL;
    if (h.T < 1 || h.P < 1 || h.d < 1 || h.d > SMC_MAX_D || h.ns < 0 || h.W < 1 || h.ndesign < 0 ||
        h.design_iters < 0 || (long long)c.J * c.N != h.P)
        return SMC_EINVAL;
    const size_t P = (size_t)h.P, d = (size_t)h.d, ns = (size_t)h.ns, T = (size_t)h.T, J = (size_t)c.J;
    const bool f32obs = m.model == SMC_EGARCH && c.precision == SMC_FP32;
    std::vector<float> obs_f(f32obs ? T : 0);
    std::vector<double> obs_d(f32obs ? 0 : T * (size_t)h.W), th(d * P), ll(P), lp(P), st(ns * P),
        gr(h.mala ? d * P : 0), a(J), as(J), pit(h.has_pit ? T : 0), dx((size_t)h.ndesign),
        dl((size_t)h.design_iters * d * d);
    std::vector<int> dr((size_t)h.ndesign);
    bool ok = get(in.f, obs_f.data(), obs_f.size() * sizeof(float)) &&
              get(in.f, obs_d.data(), obs_d.size() * sizeof(double)) &&
              get(in.f, th.data(), th.size() * sizeof(double)) && get(in.f, ll.data(), P * sizeof(double)) &&
              get(in.f, lp.data(), P * sizeof(double)) && get(in.f, st.data(), st.size() * sizeof(double)) &&
              get(in.f, gr.data(), gr.size() * sizeof(double)) && get(in.f, a.data(), J * sizeof(double)) &&
              get(in.f, as.data(), J * sizeof(double)) && get(in.f, pit.data(), pit.size() * sizeof(double)) &&
              get(in.f, dx.data(), dx.size() * sizeof(double)) && get(in.f, dr.data(), dr.size() * sizeof(int)) &&
              get(in.f, dl.data(), dl.size() * sizeof(double));
    if (!ok) return SMC_EINVAL;

    // the observations as smc_init takes them (it stores them again in the
    // same form, so the device copy is bitwise the saved one)
    std::vector<double> y(T), X;
    if (f32obs) {
        for (size_t t = 0; t < T; ++t) y[t] = (double)obs_f[t];
    } else if (m.model == SMC_LINREG) {
        X.resize(T * (size_t)m.p);
        for (size_t t = 0; t < T; ++t) {
            for (int i = 0; i < m.p; ++i) X[t * m.p + i] = obs_d[t * h.W + i];
            y[t] = obs_d[t * h.W + m.p];
        }
    } else {
        for (size_t t = 0; t < T; ++t) y[t] = obs_d[t];
    }
    // a context from the saved particles (theta in the device layout [d][P])
    cudaStream_t s = (cudaStream_t)stream;
    double* th_dev = nullptr;
    if (cudaMalloc(&th_dev, d * P * sizeof(double)) != cudaSuccess) return SMC_ENOMEM;
    std::unique_ptr<double, cudaError_t (*)(void*)> th_guard(th_dev, cudaFree);
    if (cudaMemcpy(th_dev, th.data(), d * P * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return SMC_ECUDA;
    smc_ctx* ctx = nullptr;
    smc_status stt = smc_init(&m, &c, y.data(), X.empty() ? nullptr : X.data(), h.T, th_dev, 1, stream, &ctx);
    if (stt != SMC_OK) {
        smc_free(ctx);
        return stt;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        smc_free(ctx);
        return SMC_ECUDA;
    }
    // the run state
    cudaError_t e = cudaSuccess;
    ctx->cur = 0;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(ctx->ll[0], ll.data(), P * sizeof(double));
    up(ctx->lp[0], lp.data(), P * sizeof(double));
    if (ns) up(ctx->state[0], st.data(), ns * P * sizeof(double));
    if (h.mala && ctx->grad[0]) up(ctx->grad[0], gr.data(), d * P * sizeof(double));
    up(ctx->a, a.data(), J * sizeof(double));
    up(ctx->a_score, as.data(), J * sizeof(double));
    if (h.has_pit && ctx->pit) up(ctx->pit, pit.data(), T * sizeof(double));
    up(ctx->ctl, &ctl, sizeof ctl);
    ctx->cycle = h.cycle;
    ctx->t_prev = h.t_prev;
    ctx->done = h.done;
    ctx->phi = h.phi;
    ctx->evals = h.evals;
    ctx->msteps = h.msteps;
    ctx->ppt = h.ppt;
    ctx->mut_threads = h.mut_threads;
    ctx->record = h.record;
    ctx->replay = h.replay;
    ctx->design_x = dx;
    ctx->design_R = dr;
    ctx->design_iters = h.design_iters;
    ctx->replay_iter = h.replay_iter;
    if (h.record || h.replay) {
        const int cap = h.record ? (h.design_cap > h.design_iters ? h.design_cap : h.design_iters) : h.design_iters;
        ctx->design_cap = cap;
        if (e == cudaSuccess) e = cudaMalloc(&ctx->design_L, (size_t)(cap > 0 ? cap : 1) * d * d * sizeof(double));
        if (e == cudaSuccess && !dl.empty()) up(ctx->design_L, dl.data(), dl.size() * sizeof(double));
    }
    if (e != cudaSuccess) {
        smc_free(ctx);
        return SMC_ECUDA;
    }
    *out = ctx;
    return SMC_OK;
}

extern "C" smc_status smc_describe(const smc_ctx* ctx, smc_model* m, smc_config* c, int* T)
{
    if (!ctx) return SMC_EINVAL;
    if (m) *m = ctx->model;
    if (c) *c = ctx->cfg;
    if (T) *T = ctx->T;
    return SMC_OK;
}
