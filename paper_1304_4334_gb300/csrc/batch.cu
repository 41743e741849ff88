// Batched driver: many independent simulator runs (datasets of different
// length, EGARCH models of different K and I) advanced cycle by cycle
// together.  The M phase, which carries nearly all of the work, runs as one
// persistent kernel per Metropolis iteration over every dataset's particles:
// the work items (dataset, tile of particles) sit in a queue ordered by
// decreasing cost (longest-processing-time first: T x per-observation work of
// the model) and persistent blocks pull them with an atomic counter, so
// datasets of very different T share the GPU without a tail of idle SMs.  One
// M iteration (batched covariance, persistent mutation, iteration counter) is
// a captured CUDA graph replayed R times per cycle; per-dataset parameters
// that change between cycles live in device descriptors updated once per
// cycle.  The tile size is chosen at start-up by timing the candidates
// (autotuner).  The C and S phases of each dataset are enqueued per dataset;
// all datasets share one control-block read-back per phase.  Runs whose
// mutation is MALA use the batched Langevin kernel (batch_mala.cu) in place of
// the random-walk one; one batch holds runs of one mutation kind.
#include "batch_mala.cuh"
#include "ctx.h"

#include <algorithm>
#include <cstring>
#include <new>

namespace smc {

void count_launch();

struct BatchMemberDev {
    MutateArgs a;
    int K, I, R;
};

template <int K, int I>
using PF = PolicyEgarchF32<K, I>;

// All FP32 EGARCH tiles use the same shared-memory layout.
static_assert(sizeof(MutateSmem<PF<1, 1>>) == sizeof(MutateSmem<PF<4, 4>>), "tile layouts differ");

constexpr int kBatchMaxThreads = 256;

__global__ void __launch_bounds__(kBatchMaxThreads) k_mutate_batch(const BatchMemberDev* __restrict__ mem,
                                                                   const BatchItem* __restrict__ items,
                                                                   int nitems, unsigned int* next,
                                                                   const int* iter)
{
    __shared__ MutateSmem<PF<1, 1>> sm;
    __shared__ int s_it;
    const int r = *iter;
    for (;;) {
        if (threadIdx.x == 0) s_it = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int it = s_it;
        __syncthreads();
        if (it >= nitems) break;
        const BatchItem w = items[it];
        const BatchMemberDev& bm = mem[w.member];
        if (r >= bm.R) continue;
        switch (bm.K * 8 + bm.I) {
#define SMC_BATCH_CASE(K, I)                                                                       \
    case K * 8 + I:                                                                                \
        mutate_tile<PF<K, I>>(bm.a, (uint64_t)r, w.p0, reinterpret_cast<MutateSmem<PF<K, I>>&>(sm)); \
        break;
            SMC_BATCH_CASE(1, 1) SMC_BATCH_CASE(1, 2) SMC_BATCH_CASE(1, 3) SMC_BATCH_CASE(1, 4)
            SMC_BATCH_CASE(2, 1) SMC_BATCH_CASE(2, 2) SMC_BATCH_CASE(2, 3) SMC_BATCH_CASE(2, 4)
            SMC_BATCH_CASE(3, 1) SMC_BATCH_CASE(3, 2) SMC_BATCH_CASE(3, 3) SMC_BATCH_CASE(3, 4)
            SMC_BATCH_CASE(4, 1) SMC_BATCH_CASE(4, 2) SMC_BATCH_CASE(4, 3) SMC_BATCH_CASE(4, 4)
#undef SMC_BATCH_CASE
        default: break;
        }
    }
}

__global__ void k_iter_inc(int* iter)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *iter += 1;
}

// Algorithmic per-observation work (FP32 lane ops + SFU ops) used as the
// LPT cost of a dataset: T x this.
static double obs_cost(int K, int I, int gamma)
{
    const int fp32 = 1 + (gamma ? 3 : 2) * K + K + 1 + 2 + (I == 1 ? 1 : I == 2 ? 8 : 5 * I);
    const int sfu = 1 + (I == 1 ? 0 : I == 2 ? 1 : I);
    return (double)(fp32 + sfu);
}

}  // namespace smc

struct smc_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<smc_ctx*> m;
    std::vector<BatchMemberDev> h_mem;
    std::vector<BatchMalaDev> h_mala;
    std::vector<CovJob> h_jobs;
    BatchMemberDev* d_mem = nullptr;
    BatchMalaDev* d_mala = nullptr;
    int mala = 0;                 // every run mutates by MALA
    int Kmax = 1;
    size_t mala_smem = 0;
    CovJob* d_jobs = nullptr;
    BatchItem* d_items = nullptr;
    int nitems = 0;
    int tile = 128;
    int grid = 0;
    int Gmax = 0, dmax = 0;
    unsigned int* d_next = nullptr;
    int* d_iter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int cycles = 0;
    std::string err;
};

static smc_status bset(smc_batch* b, smc_status st, const char* msg)
{
    if (b) b->err = msg;
    return st;
}

#define BCU(call)                                                                 \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            if (b) b->err = std::string(#call ": ") + cudaGetErrorString(e_);    \
            return SMC_ECUDA;                                                     \
        }                                                                         \
    } while (0)

// Work items for the current tile size, most expensive dataset first.
static smc_status build_items(smc_batch* b)
{
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const smc_ctx* a = b->m[x];
        const smc_ctx* c = b->m[y];
        return a->T * obs_cost(a->model.K, a->model.I, a->model.gamma) >
               c->T * obs_cost(c->model.K, c->model.I, c->model.gamma);
    });
    std::vector<BatchItem> items;
    for (int i : order)
        for (int p0 = 0; p0 < b->m[i]->P; p0 += b->tile) items.push_back({i, p0});
    b->nitems = (int)items.size();
    if (b->d_items) cudaFree(b->d_items);
    BCU(cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem)));
    BCU(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    int per_sm = 0;
    if (b->mala) {
        b->mala_smem = mala_batch_smem(b->Kmax, b->tile);
        BCU(mala_batch_occupancy(b->tile, b->mala_smem, &per_sm));
    } else {
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mutate_batch, b->tile, 0));
    }
    b->grid = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    return SMC_OK;
}

// Per-cycle device descriptors: current buffers, power, cycle, iterations.
static void fill_descriptors(smc_batch* b, const std::vector<int>& R)
{
    for (int i = 0; i < b->n; ++i) {
        smc_ctx* c = b->m[i];
        MutateArgs& a = b->h_mem[i].a;
        a.m = c->mdev;
        a.obs = c->obs;
        a.T = c->T;
        a.W = c->W;
        a.theta = c->theta[c->cur];
        a.ll = c->ll[c->cur];
        a.lp = c->lp[c->cur];
        a.state = c->ns ? c->state[c->cur] : nullptr;
        a.thp = c->thp;
        a.P = c->P;
        a.ns = c->ns;
        a.L = c->L;
        a.qmean = nullptr;
        a.lq = nullptr;
        a.covtile = c->covtile;
        a.covshift = c->covshift_f;
        a.ntiles = c->ntiles;
        a.phi = c->phi;
        a.seed = c->cfg.seed;
        a.cycle = (uint64_t)c->cycle;
        a.iter = 0;
        a.acc_count = &c->ctl->acc_count;
        a.pending = &c->ctl->pending;
        a.err = &c->ctl->err;
        b->h_mem[i].K = c->model.K;
        b->h_mem[i].I = c->model.I;
        b->h_mem[i].R = R[i];
        if (b->mala) {
            MalaArgs& g = b->h_mala[i].a;
            g.m = c->mdev;
            g.obs = c->obs;
            g.T = c->T;
            g.W = c->W;
            g.theta = c->theta[c->cur];
            g.ll = c->ll[c->cur];
            g.lp = c->lp[c->cur];
            g.state = c->ns ? c->state[c->cur] : nullptr;
            g.grad = c->grad[c->cur];
            g.ckpt = c->ckpt;
            g.P = c->P;
            g.ns = c->ns;
            g.L = c->L;
            g.phi = c->phi;
            g.seed = c->cfg.seed;
            g.cycle = (uint64_t)c->cycle;
            g.iter = 0;
            g.acc_count = &c->ctl->acc_count;
            g.pending = &c->ctl->pending;
            g.err = &c->ctl->err;
            b->h_mala[i].K = c->model.K;
            b->h_mala[i].I = c->model.I;
            b->h_mala[i].R = R[i];
        }
        CovJob& j = b->h_jobs[i];
        j.theta = a.theta;
        j.d = c->d;
        j.P = c->P;
        j.part = c->cov_part;
        j.G = c->cov_G;
        j.ctl = c->ctl;
        j.L = c->L;
        j.target = c->cfg.acc_target;
        j.hmin = c->cfg.hmin_tenths;
        j.hmax = c->cfg.hmax_tenths;
        j.R = R[i];
        j.tiles = c->covtile;
        j.ntiles = c->ntiles;
        j.tile_kd = c->tile_kd;
        j.shift_f = c->covshift_f;
        j.mean = c->qmean;
    }
}

static smc_status upload_descriptors(smc_batch* b)
{
    BCU(cudaMemcpyAsync(b->d_mem, b->h_mem.data(), b->n * sizeof(BatchMemberDev), cudaMemcpyHostToDevice,
                        b->stream));
    if (b->mala)
        BCU(cudaMemcpyAsync(b->d_mala, b->h_mala.data(), b->n * sizeof(BatchMalaDev), cudaMemcpyHostToDevice,
                            b->stream));
    BCU(cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), b->n * sizeof(CovJob), cudaMemcpyHostToDevice,
                        b->stream));
    return SMC_OK;
}

// One M iteration for every dataset whose iteration count is not yet reached.
static smc_status enqueue_iteration(smc_batch* b, cudaStream_t s)
{
    BCU(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned int), s));
    BCU(launch_cov_batch(b->d_jobs, b->n, b->Gmax, b->dmax, b->d_iter, s));
    if (b->mala) {
        BCU(launch_mala_batch(b->d_mala, b->d_items, b->nitems, b->d_next, b->d_iter, b->grid, b->tile,
                              b->mala_smem, s));
    } else {
        k_mutate_batch<<<b->grid, b->tile, 0, s>>>(b->d_mem, b->d_items, b->nitems, b->d_next, b->d_iter);
        count_launch();
    }
    k_iter_inc<<<1, 32, 0, s>>>(b->d_iter);
    count_launch();
    BCU(cudaGetLastError());
    return SMC_OK;
}

static smc_status capture_graph(smc_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t cs;
    BCU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BCU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    smc_status st = enqueue_iteration(b, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != SMC_OK) return st;
    BCU(e);
    b->graph = g;
    BCU(cudaGraphInstantiate(&b->exec, g, 0));
    return SMC_OK;
}

// Snapshot / restore of every member's current particles around tuning runs.
static smc_status copy_state(smc_batch* b, int to_alternate)
{
    for (smc_ctx* c : b->m) {
        const int from = to_alternate ? c->cur : c->cur ^ 1, to = from ^ 1;
        const size_t Ps = (size_t)c->P;
        BCU(cudaMemcpyAsync(c->theta[to], c->theta[from], Ps * c->d * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        BCU(cudaMemcpyAsync(c->ll[to], c->ll[from], Ps * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        BCU(cudaMemcpyAsync(c->lp[to], c->lp[from], Ps * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        if (c->ns)
            BCU(cudaMemcpyAsync(c->state[to], c->state[from], Ps * c->ns * sizeof(double),
                                cudaMemcpyDeviceToDevice, b->stream));
        if (b->mala)
            BCU(cudaMemcpyAsync(c->grad[to], c->grad[from], Ps * c->d * sizeof(double), cudaMemcpyDeviceToDevice,
                                b->stream));
        if (to_alternate) {
            BCU(cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
        } else {
            BCU(cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, b->stream));
        }
    }
    BCU(cudaStreamSynchronize(b->stream));
    return SMC_OK;
}

extern "C" {

smc_status smc_batch_init(int n, const smc_model* models, const smc_config* cfgs, const double* const* ys,
                          const int* Ts, const double* const* theta0s, void* stream, smc_batch** out)
{
    if (!out) return SMC_EINVAL;
    *out = nullptr;
    smc_batch* b = new (std::nothrow) smc_batch();
    if (!b) return SMC_ENOMEM;
    *out = b;
    if (n < 1 || !models || !cfgs || !ys || !Ts || !theta0s) return bset(b, SMC_EINVAL, "bad batch arguments");
    b->n = n;
    b->stream = (cudaStream_t)stream;
    b->mala = cfgs[0].mutation == SMC_MALA;
    for (int i = 0; i < n; ++i) {
        const smc_config& c = cfgs[i];
        if (models[i].model != SMC_EGARCH || c.precision != SMC_FP32 || c.tempering != SMC_POWER ||
            (c.mutation != SMC_RW && c.mutation != SMC_MALA) || c.stop_rule != SMC_STOP_DET)
            return bset(b, SMC_EINVAL,
                        "batched runs take FP32 EGARCH models with power tempering, random-walk or MALA "
                        "mutation and the deterministic stopping rule");
        if ((c.mutation == SMC_MALA) != (b->mala != 0))
            return bset(b, SMC_EINVAL, "the runs of one batch share one mutation kind");
        b->Kmax = std::max(b->Kmax, models[i].K);
        smc_ctx* ctx = nullptr;
        const smc_status st = smc_init(&models[i], &c, ys[i], nullptr, Ts[i], theta0s[i], 0, stream, &ctx);
        b->m.push_back(ctx);
        if (st != SMC_OK) return bset(b, st, ctx ? smc_last_error(ctx) : "member init failed");
        b->Gmax = std::max(b->Gmax, ctx->cov_G);
        b->dmax = std::max(b->dmax, ctx->d);
    }
    b->h_mem.resize(n);
    b->h_jobs.resize(n);
    if (b->mala) {
        b->h_mala.resize(n);
        BCU(cudaMalloc(&b->d_mala, n * sizeof(BatchMalaDev)));
        b->tile = kBatchMalaMaxThreads;
    }
    BCU(cudaMalloc(&b->d_mem, n * sizeof(BatchMemberDev)));
    BCU(cudaMalloc(&b->d_jobs, n * sizeof(CovJob)));
    BCU(cudaMalloc(&b->d_next, sizeof(unsigned int)));
    BCU(cudaMalloc(&b->d_iter, sizeof(int)));
    smc_status st = build_items(b);
    if (st != SMC_OK) return st;
    return capture_graph(b);
}

smc_ctx* smc_batch_member(smc_batch* b, int i) { return b && i >= 0 && i < b->n ? b->m[i] : nullptr; }

const char* smc_batch_last_error(const smc_batch* b) { return b ? b->err.c_str() : "no batch"; }

int smc_batch_tile(const smc_batch* b) { return b ? b->tile : 0; }

smc_status smc_batch_autotune(smc_batch* b, int iters, double* ms_out)
{
    if (!b) return SMC_EINVAL;
    if (iters < 1) iters = 2;
    smc_status st = copy_state(b, 1);
    if (st != SMC_OK) return st;
    std::vector<int> R(b->n, 1 << 30);
    // tune at the first cycle's target (phi = 0 until a C phase has run)
    fill_descriptors(b, R);
    st = upload_descriptors(b);
    if (st != SMC_OK) return st;
    const int cand_rw[3] = {64, 128, 256}, cand_mala[3] = {32, 64, 64};
    const int* cand = b->mala ? cand_mala : cand_rw;
    double best = 1e30;
    int best_tile = b->tile;
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    for (int ci = 0; ci < 3; ++ci) {
        const int t = cand[ci];
        b->tile = t;
        st = build_items(b);
        if (st != SMC_OK) return st;
        BCU(cudaMemsetAsync(b->d_iter, 0, sizeof(int), b->stream));
        st = enqueue_iteration(b, b->stream);   // warm-up
        if (st != SMC_OK) return st;
        BCU(cudaEventRecord(e0, b->stream));
        for (int k = 0; k < iters; ++k) {
            st = enqueue_iteration(b, b->stream);
            if (st != SMC_OK) return st;
        }
        BCU(cudaEventRecord(e1, b->stream));
        BCU(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BCU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_tile = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile = best_tile;
    st = build_items(b);
    if (st != SMC_OK) return st;
    st = copy_state(b, 0);
    if (st != SMC_OK) return st;
    if (ms_out) *ms_out = best / iters;
    return capture_graph(b);
}

smc_status smc_batch_cycle(smc_batch* b, int* n_active)
{
    if (!b) return SMC_EINVAL;
    std::vector<int> active;
    for (int i = 0; i < b->n; ++i)
        if (!b->m[i]->done) active.push_back(i);
    if (n_active) *n_active = (int)active.size();
    if (active.empty()) return SMC_EDONE;
    // C and S phases of every active run, one read-back for all
    for (int i : active) {
        smc_status st = smc_internal_enqueue_cs(b->m[i]);
        if (st != SMC_OK) return bset(b, st, smc_last_error(b->m[i]));
        st = smc_internal_enqueue_ctl_readback(b->m[i]);
        if (st != SMC_OK) return bset(b, st, smc_last_error(b->m[i]));
    }
    BCU(cudaStreamSynchronize(b->stream));
    std::vector<int> R(b->n, 0);
    std::vector<double> rss(b->n, 1.0);
    int Rmax = 0;
    for (int i : active) {
        smc_ctx* c = b->m[i];
        smc_status st = smc_internal_check(c);
        if (st != SMC_OK) return bset(b, st, smc_last_error(c));
        int forced = 0;
        smc_internal_after_cs(c, &rss[i], &forced);
        R[i] = smc_internal_R(c, rss[i]);
        Rmax = std::max(Rmax, R[i]);
    }
    // M phase: Rmax replays of the captured iteration
    fill_descriptors(b, R);
    smc_status st = upload_descriptors(b);
    if (st != SMC_OK) return st;
    BCU(cudaMemsetAsync(b->d_iter, 0, sizeof(int), b->stream));
    for (int r = 0; r < Rmax; ++r) {
        BCU(cudaGraphLaunch(b->exec, b->stream));
        for (int k = 0; k < 5; ++k) count_launch();   // kernels in the captured iteration
    }
    for (int i : active) {
        st = smc_internal_enqueue_adapt(b->m[i]);
        if (st != SMC_OK) return bset(b, st, smc_last_error(b->m[i]));
        st = smc_internal_enqueue_ctl_readback(b->m[i]);
        if (st != SMC_OK) return bset(b, st, smc_last_error(b->m[i]));
    }
    BCU(cudaStreamSynchronize(b->stream));
    for (int i : active) {
        smc_ctx* c = b->m[i];
        st = smc_internal_check(c);
        if (st != SMC_OK) return bset(b, st, smc_last_error(c));
        st = smc_internal_after_m(c, c->T, R[i], c->T, c->phi, rss[i], nullptr);
        if (st != SMC_OK) return bset(b, st, smc_last_error(c));
    }
    b->cycles += 1;
    return SMC_OK;
}

smc_status smc_batch_run(smc_batch* b, int max_cycles, int* ncycles)
{
    if (!b) return SMC_EINVAL;
    int k = 0;
    for (;;) {
        if (max_cycles > 0 && k >= max_cycles) break;
        int act = 0;
        const smc_status st = smc_batch_cycle(b, &act);
        if (st == SMC_EDONE) break;
        if (st != SMC_OK) {
            if (ncycles) *ncycles = k;
            return st;
        }
        ++k;
    }
    if (ncycles) *ncycles = k;
    return SMC_OK;
}

smc_status smc_batch_reset(smc_batch* b, const double* const* theta0s, int on_device, uint64_t seed)
{
    if (!b || !theta0s) return SMC_EINVAL;
    for (int i = 0; i < b->n; ++i) {
        const smc_status st = smc_reset(b->m[i], theta0s[i], on_device, seed + (uint64_t)i);
        if (st != SMC_OK) return bset(b, st, smc_last_error(b->m[i]));
    }
    b->cycles = 0;
    return SMC_OK;
}

smc_status smc_batch_totals(smc_batch* b, double* evals, int64_t* metropolis_steps, int* cycles)
{
    if (!b) return SMC_EINVAL;
    double e = 0.0;
    int64_t ms = 0;
    for (smc_ctx* c : b->m) {
        e += c->evals;
        ms += c->msteps;
    }
    if (evals) *evals = e;
    if (metropolis_steps) *metropolis_steps = ms;
    if (cycles) *cycles = b->cycles;
    return SMC_OK;
}

void smc_batch_free(smc_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (smc_ctx* c : b->m) smc_free(c);
    void* ptrs[] = {b->d_mem, b->d_mala, b->d_jobs, b->d_items, b->d_next, b->d_iter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

}  // extern "C"
