// Internal: the simulator context and the driver steps shared by the single-run
// and batched drivers (api.cu, batch.cu).  Not part of the C ABI.
#pragma once

#include "../../include/smc.h"
#include "kernels.cuh"
#include "mala.cuh"
#include "phase.cuh"

#include <string>
#include <utility>
#include <vector>

using namespace smc;

struct smc_ctx {
    smc_model model;
    smc_config cfg;
    ModelDev mdev;
    int T = 0, P = 0, d = 0, ns = 0, W = 1;
    cudaStream_t stream = nullptr;
    // observations
    void* obs = nullptr;             // float[T] (FP32 EGARCH) or double[T*W]
    // particles, double-buffered for the S-phase gather
    double* theta[2] = {nullptr, nullptr};
    double* ll[2] = {nullptr, nullptr};
    double* lp[2] = {nullptr, nullptr};
    double* state[2] = {nullptr, nullptr};
    double* grad[2] = {nullptr, nullptr};  // MALA: likelihood gradient [d][P]
    void* ckpt = nullptr;                  // MALA: recursion checkpoints
    int cur = 0;
    double* thp = nullptr;           // proposal scratch [d][P]
    double* logw = nullptr;          // [P] data tempering log weights
    double* g = nullptr;             // [3][P] test functions
    // per-group estimators
    double* a = nullptr;             // [J]
    double* a_score = nullptr;       // [J] log score accumulators (cycles after the burn-in)
    double* pit = nullptr;           // [T] probability integral transforms (nullable)
    double* lw = nullptr;            // [J]
    double* gstat = nullptr;         // [J][3]
    int32_t* idx = nullptr;          // [P]
    double* cov_part = nullptr;
    int cov_G = 0;
    double* search_part = nullptr;
    double* cd_part = nullptr;       // [G][kCdataChunk][3] data-tempering statistics
    double* cd_end = nullptr;        // [1 + ns][P] data tempering: the chunk's sum and end state (statistics pass)
    double* mom_part = nullptr;      // [nf][J][2]
    double* mom_out = nullptr;       // [nf][4]
    double* ml_out = nullptr;        // [3]
    double* L = nullptr;             // [d][d]
    double* qmean = nullptr;         // [d] pooled mean of the particles at the last covariance
                                     // (independent-sampler proposal mean; shift of the tiles)
    float* covtile = nullptr;        // [kD + kD(kD+1)/2][ntiles] mutation-kernel covariance tile sums
    float* covshift_f = nullptr;     // [d] the tiles' shift (pooled mean rounded to FP32)
    int tile_kd = 0;                 // the mutation policy's parameter bound kD
    double* cov_tot = nullptr;       // [nacc] combined tile sums
    unsigned int* cov_counter = nullptr;  // last-block counter of the covariance reduction (zero between launches)
    int ntiles = 0;
    bool tiles_ready = false;        // covtile holds the current particles' sums
    double* lq = nullptr;            // [P] independent sampler: log q of the current particles
    double** gather_ptrs = nullptr;  // [2][nrows] device row-pointer tables
    int gather_rows = 0;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;         // pinned, two blocks: [0] the latest read-back, [1] the M phase's (pipelined runs)
    // run state
    int cycle = 0, t_prev = 0, done = 0;
    int cd_chunks = 0;   // data tempering: chunks the last cycle's C phase took (batch size only)
    double phi = 0.0;
    int64_t msteps = 0;
    double evals = 0.0;
    uint64_t h2d = 0, d2h = 0;
    // Algorithm 3 (hybrid): design recording / replay
    int record = 0, replay = 0;
    std::vector<double> design_x;        // t_l (data) or phi_l (power) per cycle
    std::vector<int> design_R;           // Metropolis iterations per cycle
    double* design_L = nullptr;          // device, [iterations][d][d]
    int design_cap = 0;                  // capacity of design_L in iterations
    int design_iters = 0;                // iterations recorded, or loaded for replay
    int replay_iter = 0;                 // next factor to use in replay
    // mutation launch shape (FP32 EGARCH): particles per thread and block size
    int ppt = 1, mut_threads = kMutThreads;
    // profiling
    int profile = 0;
    double mutate_ms = 0.0;
    uint64_t mutate_launches = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::string err;
};


// Driver steps (api.cu).  "enqueue" steps only enqueue work on the context's
// stream; "after" steps read the control block copied back by the last sync.
smc_status smc_internal_enqueue_cs(smc_ctx* ctx);          // power tempering C + S phases
smc_status smc_internal_enqueue_ctl_readback(smc_ctx* ctx);
smc_status smc_internal_check(smc_ctx* ctx);               // device error bits after a sync
void smc_internal_after_cs(smc_ctx* ctx, double* rss, int* forced);
int smc_internal_R(const smc_ctx* ctx, double rss);
smc_status smc_internal_enqueue_adapt(smc_ctx* ctx);
smc_status smc_internal_after_m(smc_ctx* ctx, int t_l, int R, int Tm, double phim, double rss,
                                smc_cycle_info* info);
