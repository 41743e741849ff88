// C, S and estimator kernels around the M phase, and the device-resident
// control block that lets a whole cycle run without host round trips between
// its kernels.
#pragma once

#include "recursion.cuh"

namespace smc {

// Device-resident control state of a run.
struct Ctl {
    // M phase: step size in tenths (Section 3.3) and acceptance bookkeeping.
    int h_tenths;
    int pending;                    // an acceptance count awaits its h update
    unsigned long long acc_count;   // accepted proposals of the pending iteration
    double acc_sum;                 // sum of acceptance rates in this cycle
    int acc_n;                      // iterations in this cycle
    // C phase, power tempering: k-ary search state.
    double llmax, lo, hi, dphi, rss, phi;
    int pass, done, last;
    // C phase, data tempering: observations to absorb from the current chunk,
    // the chunk (1-based number within the cycle) that contains the stopping
    // observation or 0, and whether the stop was forced (date of interest or
    // T with RSS >= D1).  Chunks numbered after cd_found do nothing.
    int cd_stop, cd_found, cd_forced;
    // RNE stopping rule.
    double mean_rne;
    // Estimators (Section 4.2): log wtilde accumulates log of J^-1 sum_j wbar_j(l-1).
    double ltilde;
    int err;
};

// ---- launchers (phase.cu) ----
int device_sm_count();

// Covariance: partial sums per block (part: [G + 1][nacc] doubles, the last
// row receiving the totals), then one block per total whose last finisher
// applies the pending step-size update and factors h^2 V.  counter: a device
// word that is zero before the call and zero again after it.
int cov_grid(int P);
cudaError_t launch_cov(const double* theta, int d, int P, double* part, int G, unsigned int* counter,
                       Ctl* ctl, int fixed_h_tenths, double acc_target, int hmin, int hmax, double* mean,
                       double* cov, double* L, cudaStream_t s, float* mean_f = nullptr);
// From the mutation kernel's 32-particle tile sums (entry-major
// [kD + kD(kD+1)/2][ntiles], values shifted by shift_f): combine in FP64, then
// the same final step; the pooled mean goes to mean (FP64) and, rounded, back
// into shift_f (the next tiles' shift).
cudaError_t launch_cov_tiles(const float* tiles, int ntiles, int tile_kd, int d, int P, double* tot,
                             unsigned int* counter, float* shift_f, double* mean, Ctl* ctl, int fixed_h_tenths,
                             double acc_target, int hmin, int hmax, double* L, cudaStream_t s);
// Batched form: one covariance job per particle set, skipped once the
// device iteration counter reaches the job's iteration count R.
struct CovJob {
    const double* theta;
    int d, P;
    double* part;     // (G + 1) x (d + d(d+1)/2)
    int G;
    Ctl* ctl;
    double* L;
    double target;
    int hmin, hmax;
    int R;
    const float* tiles;   // mutation tile sums [kD + kD(kD+1)/2][ntiles] (nullable)
    int ntiles, tile_kd;
    float* shift_f;       // [d] the tiles' shift: the pooled mean rounded, rewritten by each final step
    double* mean;         // [d] pooled mean
};
cudaError_t launch_cov_batch(const CovJob* jobs, int n, int Gmax, int dmax, const int* iter, cudaStream_t s);

// Applies a pending acceptance count to h (end of an M phase).
cudaError_t launch_adapt_h(Ctl* ctl, int P, double acc_target, int hmin, int hmax, cudaStream_t s);

// Power-tempering search; part sized search_part_len(P) doubles, whose first
// search_bar_bytes() bytes (grid-barrier words) are zero before the first
// call and are left zero by every call that completes.
int search_grid(int P);
size_t search_part_len(int P);
size_t search_bar_bytes();
cudaError_t launch_power_search(const double* ll, int P, double d1, int passes, double* part,
                                Ctl* ctl, cudaStream_t s);

// Replay (Algorithm 3): set the increment to reach a recorded power.
cudaError_t launch_set_power(Ctl* ctl, double phi_target, cudaStream_t s);

// S phase: per group weights, log-mean weight (a_j, lw_j), resampling, then gather.
// mode 0: weights from ctl->dphi * ll; mode 1: from logw; mode 2: w given directly.
struct SelectArgs {
    int mode;
    const double* ll;
    const double* logw;
    const double* w;
    int J, N;
    int scheme;       // 0 residual, 1 multinomial, 2 stratified, 3 systematic
    uint64_t seed, cycle;
    double* a;        // [J] += log wbar_j (modes 0, 1)
    double* a_score;  // [J] += log wbar_j too (nullable: cycles before the burn-in)
    double* lw;       // [J] log wbar_j of this cycle (modes 0, 1)
    double* gstat;    // [J][3] (max log w, sum w, sum w^2) of this cycle (modes 0, 1)
    int32_t* idx;     // [J*N]
    Ctl* ctl;
    int* err;
};
size_t select_smem(int N);
cudaError_t launch_select(const SelectArgs& a, cudaStream_t s);

struct GatherArgs {
    const int32_t* idx;
    int N, P;
    int nrows;                 // rows of length P to gather (theta's d rows first)
    const double* const* src;  // device array of nrows row pointers
    double* const* dst;        // device array of nrows row pointers
    // Covariance tile sums of the gathered particles for the next M phase's
    // first covariance step (nullable): the same 32-particle tiles and layout
    // as the mutation kernel's, about the shift theta of the particle placed
    // in slot 0 (rounded to FP32), which is also written to covshift.
    float* covtile = nullptr;
    float* covshift = nullptr;
    int ntiles = 0, d = 0, tile_kd = 0;
};
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);

// Data tempering: combine the per-block statistics of one chunk and choose
// the stopping observation (first s with RSS(s) < D1, a date of interest, or T).
struct ForceDates {
    int n;
    int t[65];   // dates of interest and the burn-in date
};
// Chunk scratch of the data-tempering C phase: per block and observation
// (max log w, sum w, sum w^2), then the stop search's tail (zeroed once).
size_t cdata_part_len(int G);
cudaError_t launch_cdata_select(double* part, int G, int B, int s0, int T, int P, double d1,
                                const ForceDates& fd, Ctl* ctl, int seq, cudaStream_t s);
cudaError_t launch_pit_final(const double* part, int G, int B, int s0, const Ctl* ctl, double* pit, int seq,
                             cudaStream_t s);

// After the S phase: pooled RSS at the chosen power, log wtilde, phi update.
cudaError_t launch_cycle_close(const double* gstat, const double* lw, int J, int N, int power,
                               Ctl* ctl, cudaStream_t s);

// Test functions g1..g3 (Section 5.2) into g[3][P].
cudaError_t launch_testfn(const ModelDev& m, int precision, const double* theta,
                          const double* state, int P, double* g, cudaStream_t s);
// Group moments of nf rows of g ([nf][J*N]) into out[nf][4] (device); optional
// mean RNE of rows [rne_from, nf) into ctl->mean_rne.
cudaError_t launch_moments(const double* g, int nf, int J, int N, double* part, double* out,
                           Ctl* ctl, int rne_from, cudaStream_t s);
// log ML and NSE from a[J]; out[0..2] = log wbar, NSE, log wtilde (from ctl, if given).
cudaError_t launch_ml(const double* a, int J, const Ctl* ctl, double* out, cudaStream_t s);

}  // namespace smc
