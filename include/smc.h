/*
 * smc.h - C ABI of libsmc.so, a GB300 (sm_103a) implementation of the adaptive
 * sequential posterior simulator of Durham & Geweke, "Adaptive Sequential
 * Posterior Simulators for Massively Parallel Computing Environments" (2013).
 *
 * The simulator (Algorithm 2 with the specifics of Section 3.3) moves J groups
 * of N particles from the prior to the posterior in cycles of three phases:
 *   C (correction):  reweight by the next slice of likelihood; the slice ends
 *                    when the relative sample size RSS = ESS / (J N) drops
 *                    below D1 (Section 3.3, "C phase termination").  Two forms:
 *                    SMC_DATA adds observations one at a time (Algorithm 1,
 *                    (C_phase_compute)); SMC_POWER raises the full-sample
 *                    likelihood to the next power phi, found by a k-ary
 *                    bisection so that RSS reaches D1.
 *   S (selection):   residual (default) or multinomial resampling within each
 *                    group (Section 3.3, "Resampling method").
 *   M (mutation):    Gaussian random-walk Metropolis with Sigma = h^2 V,
 *                    V the pooled particle covariance, h adapted toward an
 *                    acceptance target (Section 3.3, "Metropolis steps"); the
 *                    number of iterations follows the deterministic or the
 *                    RNE-based rule ("M phase Termination").
 * The log marginal likelihood and its numerical standard error come from the
 * per-group products of mean weights (Section 4.2, (ML_se)); posterior moments
 * with NSE and RNE from the between-group variance (Section 2.3, (NSE_def)).
 *
 * Conventions for every function below:
 *   - Return value: SMC_OK or an error code; nothing is thrown across the ABI.
 *     The context-taking calls keep a message for smc_last_error().
 *   - "device" pointers are CUDA device addresses on the current device; "host"
 *     pointers are ordinary memory.  Inputs are copied in; the caller keeps
 *     ownership of everything it passes.  A context owns all device memory it
 *     allocates and releases it in smc_free().
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; functions that return host values
 *     synchronise that stream before returning.
 *   - Particle arrays on the device are structure-of-arrays: theta is [d][P]
 *     (parameter-major, P = J N), state is [K+1][P].  Host particle arrays
 *     are particle-major [P][d].
 *   - There is no CPU fallback: without a usable GPU every call that computes
 *     returns SMC_ECUDA.
 */
#ifndef SMC_H
#define SMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SMC_MAX_D 32      /* free parameters per particle */
#define SMC_MAX_FORCE 64  /* dates of interest */
#define SMC_MAX_N 8192    /* particles per group */

typedef enum {
    SMC_OK = 0,
    SMC_EINVAL = 1,       /* invalid argument (message in smc_last_error) */
    SMC_ENOMEM = 2,       /* device or host allocation failed */
    SMC_ECUDA = 3,        /* CUDA runtime error, or no usable GPU */
    SMC_EDEGENERATE = 4,  /* a group has zero total weight */
    SMC_ENONFINITE = 5,   /* non-finite input data */
    SMC_ETIMEOUT = 6,     /* a bounded device wait ran out */
    SMC_EDONE = 7         /* the run has already reached the full posterior */
} smc_status;

enum { SMC_EGARCH = 0, SMC_LINREG = 1 };
enum { SMC_FP64 = 0, SMC_FP32 = 1 };
enum { SMC_DATA = 0, SMC_POWER = 1 };
enum { SMC_RW = 0, SMC_MALA = 1, SMC_INDEP = 2 };
enum { SMC_RESIDUAL = 0, SMC_MULTINOMIAL = 1, SMC_STRATIFIED = 2, SMC_SYSTEMATIC = 3 };
enum { SMC_STOP_DET = 0, SMC_STOP_RNE = 1 };

/* Model description (plain data).
 * EGARCH(K, I) of Section 5.1, (EGARCH_mod1)-(EGARCH_mod2) with the normal
 * mixture (normal_mixture); parameters are the transformed theta of Table 1,
 * laid out as theta_1, theta_2, theta_3k (k = 1..K), theta_4k, [theta_5k if
 * gamma], [theta_6i, theta_7i, theta_8i (i = 1..I) if I >= 2].  With I = 1 the
 * normalisation (EGARCH_normalization) fixes the mixture, so it carries no
 * parameters.  eps0_zero selects v_k1 = -beta_k (2/pi)^1/2 instead of the
 * default v_k1 = 0 (no shock before the first observation).
 * LINREG: y_t = x_t' beta + e_t, e_t ~ N(0, sigma^2) with sigma known
 * (a conjugate check model; theta = beta, p <= 7).
 * Priors are independent Gaussians on the free parameters, truncated below at
 * prior_lo (-inf for none); the log prior is the density kernel of
 * Condition 1 (truncation constants omitted).
 * n_free = 0 means all d_full parameters are free; otherwise only
 * free_idx[0..n_free) move and the rest stay at theta_fixed. */
typedef struct {
    int model;
    int K, I, gamma, eps0_zero;
    int p;
    double sigma;
    int d_full;                       /* filled by smc_model_egarch/linreg */
    int n_free;
    int free_idx[SMC_MAX_D];
    double theta_fixed[SMC_MAX_D];
    double prior_mean[SMC_MAX_D];     /* over the free parameters, in order */
    double prior_sd[SMC_MAX_D];
    double prior_lo[SMC_MAX_D];
} smc_model;

/* Fills an EGARCH(K, I) description with the priors of Table 1
 * (K in 1..4, I in 1..4; gamma = 0 drops theta_5k). */
smc_status smc_model_egarch(smc_model* m, int K, int I, int gamma);
/* Fills a LINREG description; prior_mean/prior_sd are host arrays of p. */
smc_status smc_model_linreg(smc_model* m, int p, double sigma, const double* prior_mean,
                            const double* prior_sd);
/* Number of parameters each particle carries. */
int smc_model_dim(const smc_model* m);

/* Simulator settings.  smc_config_default gives the defaults of Section 3.3:
 * D1 = 0.5, D2 = 0.2, Rbar = 7, kappa = 3, E1 = 0.35, E2 = 0.90, Rmax = 100,
 * h0 = 0.5 in steps of 0.1 within [0.1, 1.0], acceptance target 0.25,
 * residual resampling, random-walk mutation, deterministic stopping rule,
 * power tempering, FP32 recursion. */
typedef struct {
    int J, N;                 /* groups x particles per group (N <= SMC_MAX_N) */
    int precision;            /* SMC_FP32: recursion in FP32 with FP64 log-likelihood,
                                 log weights and estimators; SMC_FP64: all FP64 */
    int tempering;            /* SMC_POWER | SMC_DATA */
    int mutation;             /* SMC_RW | SMC_MALA (Langevin proposal using the adjoint gradient)
                                 | SMC_INDEP (Section 3.3's independent Gaussian sampler:
                                 proposal N(mean, V) from the pooled mean and variance of
                                 the population; no step size; no hybrid record/replay) */
    int resampler;            /* SMC_RESIDUAL (default) | SMC_MULTINOMIAL, or the paper's
                                 experimental SMC_STRATIFIED | SMC_SYSTEMATIC */
    double d1, d2;
    int stop_rule;            /* SMC_STOP_DET | SMC_STOP_RNE */
    int rbar, kappa, rmax;
    double e1, e2;
    int h0_tenths, hmin_tenths, hmax_tenths;
    double acc_target;
    int h_reset_each_cycle;
    int n_force;              /* data tempering: dates of interest (1-based) */
    int force_dates[SMC_MAX_FORCE];
    int search_passes;        /* power tempering: k-ary passes (32 candidates each) */
    uint64_t seed;
    int burnin;               /* data tempering: b > 0 ends a cycle at t = b and makes
                                 smc_log_score report log p(y_{b+1:T} | y_1:b) (Section 4.1;
                                 0 = none, b < T) */
    int pit;                  /* data tempering: 1 records the probability integral
                                 transform of every observation (smc_pit) */
} smc_config;

void smc_config_default(smc_config* c);

/* Per-cycle report of smc_cycle. */
typedef struct {
    int cycle;                /* l, 1-based */
    int t;                    /* data tempering: t_l; power tempering: T */
    double phi;               /* power reached after the C phase (1 in data tempering) */
    double rss;               /* RSS at the end of the C phase */
    int R;                    /* Metropolis iterations run in the M phase */
    int h_tenths;             /* step size after the M phase */
    double acc_rate;          /* mean acceptance rate over the M phase */
    double evals;             /* particle x observation likelihood evaluations in the M phase */
    int done;                 /* 1 once the full posterior is reached */
} smc_cycle_info;

typedef struct smc_ctx smc_ctx;

/* Creates a context and runs step 1 of Algorithm 1: the given prior draws
 * theta0 (P x d, particle-major, host; or [d][P] device when theta0_on_device)
 * get their log prior and, in power tempering, their full-sample log
 * likelihood.  y: host array of T observations (EGARCH); X: host T x p
 * regressors (LINREG, with y).  Non-finite y or X gives SMC_ENONFINITE. */
smc_status smc_init(const smc_model* m, const smc_config* c, const double* y, const double* X,
                    int T, const double* theta0, int theta0_on_device, void* stream,
                    smc_ctx** out);

/* One C + S + M cycle (Algorithm 2).  Returns SMC_EDONE if the previous cycle
 * already reached t = T (data) or phi = 1 (power). */
smc_status smc_cycle(smc_ctx* ctx, smc_cycle_info* info);

/* Cycles until the full posterior is reached (at most max_cycles, 0 = no cap).
 * info (nullable) receives the last cycle's report; ncycles (nullable) the
 * number of cycles run by this call.  The next cycle's C phase (power
 * tempering: with its S phase; data tempering: its first batch of 32-
 * observation chunks) is enqueued behind each M phase, so that one host
 * synchronisation serves both; the kernels, their order and the results are
 * those of repeated smc_cycle calls, bit for bit. */
smc_status smc_run(smc_ctx* ctx, int max_cycles, smc_cycle_info* info, int* ncycles);

/* Restarts the run from new prior draws (same layout rules as smc_init),
 * keeping the context's buffers and observations; seed replaces the
 * configured seed.  No device memory is allocated. */
smc_status smc_reset(smc_ctx* ctx, const double* theta0, int theta0_on_device, uint64_t seed);

/* Totals since the last smc_init/smc_reset: cycles, Metropolis iterations and
 * M-phase particle x observation likelihood evaluations (host outputs,
 * nullable). */
smc_status smc_run_totals(smc_ctx* ctx, int* cycles, int64_t* metropolis_steps, double* evals);

/* Bytes this context has copied host->device and device->host since it was
 * created (host outputs, nullable). */
smc_status smc_transfer_bytes(smc_ctx* ctx, uint64_t* h2d, uint64_t* d2h);

/* log wbar^(J,N) with its working NSE from (ML_se), and log wtilde^(J,N)
 * (Section 4.2).  Host outputs; any may be NULL. */
smc_status smc_log_ml(smc_ctx* ctx, double* log_ml, double* nse, double* log_ml_tilde);

/* Per-group state of the estimators of Section 4.2 (host outputs of J doubles,
 * nullable; synchronises): a[j] = the sum over the completed cycles of
 * log wbar_j(l-1), the group's log marginal-likelihood accumulator, so that
 * smc_log_ml's log wbar^(J,N) = log J^-1 sum_j exp(a_j); lw[j] = log wbar_j(l-1)
 * of the last completed cycle, the log of the mean over the group's N
 * particles of the weights w_jn(l-1) that its C phase formed ((C_phase_compute);
 * in power tempering w = exp(dphi l(theta))). */
smc_status smc_group_estimators(smc_ctx* ctx, double* a, double* lw);

/* Posterior moments at the current particles: for each free parameter and,
 * for EGARCH, the test functions g1 (log volatility), g2 (E eps^3) and g3
 * (P(Y_t+1 < -0.03)) of Section 5.2: mean, s.d., NSE (NSE_def) and RNE.
 * out: host array of nf x 4 with nf = d (+3 for EGARCH); *nf receives nf. */
smc_status smc_moments(smc_ctx* ctx, double* out, int* nf);

/* Copies the particles to host arrays (particle-major theta [P][d]; loglik,
 * logprior [P]; state [P][K+1]).  Any pointer may be NULL. */
smc_status smc_get_particles(smc_ctx* ctx, double* theta, double* loglik, double* logprior,
                             double* state);

/* Algorithm 3 (hybrid).  Step 1 runs the adaptive simulator while recording
 * its design: for each cycle its end x_l (t_l in data tempering, phi_l in
 * power tempering) and iteration count R_l, and for each Metropolis iteration
 * the lower Cholesky factor of Sigma_lr = h^2 V (Section 3.3 lists these as
 * the design elements to keep).  Step 2 replays that design in a new context
 * (new prior draws and seed): no RSS search, covariance or step-size
 * adaptation, so the run is Algorithm 1 with fixed {t_l, lambda_l}.
 * smc_design_record: call before the first cycle; max_iterations bounds the
 * number of iterations recorded (device memory d*d doubles each).
 * smc_design_get: x[ncycles], R[ncycles], L[niterations][d][d] (host,
 * nullable), sizes from smc_design_size.  smc_design_replay: host arrays of
 * the same layout; call before the first cycle (random-walk runs only). */
smc_status smc_design_record(smc_ctx* ctx, int max_iterations);
smc_status smc_design_size(smc_ctx* ctx, int* ncycles, int* niterations);
smc_status smc_design_get(smc_ctx* ctx, double* x, int* R, double* L);
smc_status smc_design_replay(smc_ctx* ctx, int ncycles, const double* x, const int* R, const double* L);

/* Launch shape of the M-phase mutation kernel.  For FP32 EGARCH random-walk
 * runs a thread can carry two particles, whose recursions run side by side in
 * Blackwell's paired FP32 instructions (one issue slot for both; results
 * bitwise those of one particle per thread).
 * smc_autotune times `iters` Metropolis iterations of each candidate shape
 * (random walk: 1 particle x 128, 64 or 32 threads per block, and the
 * balanced block below; FP32 EGARCH also 2 particles x 32, 64, 128 threads and
 * balanced, the pair's recursions in packed FP32x2 instructions; MALA: 1 x 128
 * only) on a snapshot of the particles, restores them, and keeps the fastest;
 * outputs (host, nullable): the shape and its time per iteration.  Results do
 * not depend on the shape.  The balanced block spreads the particles' warps
 * as evenly as possible over the SMs: 32 ceil(W / (S k)) threads for W warps,
 * S SMs and the fewest blocks per SM k that keep it within 224 threads.
 * smc_set_launch_shape sets one directly: ppt 1 or 2 (2 for the FP32 EGARCH
 * random walk only), threads a multiple of 32 from 32 to 224; SMC_EINVAL
 * otherwise. */
smc_status smc_autotune(smc_ctx* ctx, int iters, int* ppt, int* threads, double* ms_per_iteration);
smc_status smc_set_launch_shape(smc_ctx* ctx, int ppt, int threads);

/* Log score log p(y_{b+1:T} | y_1:b) (Section 4.1, the predictive likelihood
 * after the burn-in b of the config): the group-product estimator over the
 * cycles that start at or after b, with its NSE by (ML_se).  Valid once the
 * run is complete; SMC_EINVAL without a burn-in.  Synchronises. */
smc_status smc_log_score(smc_ctx* ctx, double* log_score, double* nse);

/* Probability integral transform of y_s, s = 1..T (Section 4.1), for a context
 * created with pit = 1: the C-phase weighted share, weights w_jn(s-1), of
 * auxiliary draws Y_s ~ p(Y_s | y_1:s-1, theta_jn) with Y_s <= y_s.  The draw
 * of particle jn is its standardized shock from the Philox block at counter
 * (particle, s, 0, 4 << 32): uniform 0 picks mixture component i (first i with
 * u < p_1 + .. + p_i), uniforms 1 and 2 a Box-Muller normal z, shock
 * mu_i + sigma_i z (LINREG: z).  out: host [T]; observations not yet reached
 * are NaN.  Synchronises. */
smc_status smc_pit(smc_ctx* ctx, double* out, int T);

/* Prior simulation (Table 1) on the device: theta (device [d][P]) gets P
 * draws of the model's free parameters, theta_i = prior_mean_i + prior_sd_i z
 * with z standard normal, components with a finite prior_lo redrawn until they
 * are inside (truncation by rejection; after 64 rejected attempts the bound
 * itself).  Component i of particle n at attempt a is normal i % 4 of the
 * Philox4x64-10 block at counter (n, a, 0, 5 << 32 | i / 4), key (seed, 0),
 * by Box-Muller on the 53-bit uniform pairs (0, 1) and (2, 3) (cosine for the
 * even, sine for the odd normal).  The result is a valid theta0 for smc_init
 * with theta0_on_device = 1.  Asynchronous on `stream`. */
smc_status smc_draw_prior(const smc_model* m, uint64_t seed, int P, double* theta, void* stream);

/* Checkpoint and resume between cycles.  smc_save writes everything a run
 * carries across a cycle boundary to `path`: the model, the settings, the
 * observations, the current particles (theta, log likelihood, log prior,
 * recursion state, MALA gradient), the per-group log-ML and log-score
 * accumulators, the PIT values, the device control block (step size, power,
 * log wtilde, acceptance bookkeeping), the cycle count and the hybrid design
 * being recorded or replayed.  Call it between smc_cycle calls (it
 * synchronises the stream).  smc_load creates a context from such a file on
 * `stream` (the caller frees it with smc_free); later smc_cycle calls continue
 * the saved run exactly, the random numbers being counter-based.  SMC_EINVAL
 * for an unreadable or inconsistent file (written by another build of the
 * library, for instance); SMC_ECUDA / SMC_ENOMEM for device failures.
 * smc_describe copies a context's model, settings and observation count
 * (each output nullable). */
smc_status smc_save(smc_ctx* ctx, const char* path);
smc_status smc_load(const char* path, void* stream, smc_ctx** out);
smc_status smc_describe(const smc_ctx* ctx, smc_model* m, smc_config* c, int* T);

/* Failure-detection self-test: one block runs the library's bounded mbarrier
 * wait (the one guarding every staged-observation copy) with a limit of
 * limit_ns (0 < limit_ns <= 2 s) on a barrier that is completed only when
 * `complete` is nonzero.  Returns SMC_ETIMEOUT when the wait ran out (the
 * kernel then returns normally and the context stays usable), SMC_OK when it
 * completed, SMC_EINVAL for a bad limit.  Synchronises the stream.  The paper
 * has no counterpart; it exists so that the timeout path can be exercised
 * without faulting or hanging the device. */
smc_status smc_wait_selftest(uint64_t limit_ns, int complete, void* stream);

/* Peak rates of the ALU pipes of the current device, measured by a
 * microbenchmark (the paper has no counterpart: the likelihood kernels are
 * bound by plain FP32/SFU arithmetic and instruction issue, and their roofline
 * needs these rates on the part at hand).  Each test runs one block of 1024
 * threads on every SM, each thread eight independent chains of one operation.
 * Outputs (host struct): lane operations per SM and clock for ffma
 * (fma.rn.f32), ffma2 (fma.rn.f32x2, two lane operations per instruction),
 * ex2 and lg2 (ex2/lg2.approx.ftz.f32, each with one FP32 operand fix-up on
 * another pipe) and dfma (fma.rn.f64); issue = warp instructions per SM and
 * clock with an FFMA and a logic operation on its result in turn; sm_mhz = the SM clock during
 * the tests (cycle counter over the global nanosecond timer); sms = SM count;
 * ffma_mix = FP32 lane operations per SM and clock with an FFMA2 and an FFMA
 * on independent chains in turn.
 * Takes about 10 ms; allocates and frees a few bytes of device memory;
 * synchronises `stream`.  SMC_ECUDA without a usable GPU. */
typedef struct {
    int sms;
    double ffma, ffma2, ex2, lg2, dfma, issue;
    double sm_mhz;
    double ffma_mix;
} smc_peak_rates;
smc_status smc_peaks(smc_peak_rates* out, void* stream);

/* Number of kernel launches this library has issued in this process. */
uint64_t smc_launch_count(void);

/* Total device time (ms, CUDA events on the context's stream) and launch count
 * of the timed M-phase mutation launches since the context was created or the
 * timer last reset.  smc_profile(ctx, 1) times every launch; smc_profile(ctx, 2)
 * times the first launch of each M phase only, so that the covariance steps
 * after the other launches keep their programmatic dependent launch (a recorded
 * event between two kernels serialises them); 0 turns timing off.  Other
 * values: SMC_EINVAL. */
smc_status smc_profile(smc_ctx* ctx, int enable);
smc_status smc_mutate_time(smc_ctx* ctx, double* ms, uint64_t* launches, int reset);

void smc_free(smc_ctx* ctx);
const char* smc_last_error(const smc_ctx* ctx);
const char* smc_status_str(smc_status s);

/* ---------------------------------------------------------------------------
 * Batched runs: n independent simulator runs (datasets of different length T,
 * EGARCH models of different K and I; FP32, power tempering, deterministic
 * stopping rule; all random walk or all MALA) advanced together cycle by
 * cycle.  Each run is Algorithm 2 as in smc_cycle and keeps its own particles,
 * seed and adaptation; the batch shares the M-phase launches: one persistent
 * kernel per Metropolis iteration processes every run's particles from a work
 * queue ordered by decreasing cost (T x per-observation work), and one
 * iteration (batched covariance + persistent mutation) is a captured CUDA
 * graph.  Results equal those of the same runs done one at a time, bit for
 * bit.  SMC_EINVAL for other settings or for a batch mixing mutation kinds.
 * ------------------------------------------------------------------------- */
typedef struct smc_batch smc_batch;

/* ys[i]: host observations of run i (Ts[i] of them); theta0s[i]: host prior
 * draws [P_i][d_i].  On error *out is still set (free it with smc_batch_free). */
smc_status smc_batch_init(int n, const smc_model* models, const smc_config* cfgs, const double* const* ys,
                          const int* Ts, const double* const* theta0s, void* stream, smc_batch** out);
/* Times `iters` M iterations for each candidate tile (random walk: 64, 128,
 * 256 particles per work item; MALA: 32, 64) on a snapshot of the particles
 * (restored afterwards) and keeps the fastest; ms_per_iteration (host,
 * nullable) gets its time. */
smc_status smc_batch_autotune(smc_batch* b, int iters, double* ms_per_iteration);
/* One cycle of every unfinished run; SMC_EDONE when all are done. */
smc_status smc_batch_cycle(smc_batch* b, int* n_active);
smc_status smc_batch_run(smc_batch* b, int max_cycles, int* ncycles);
/* Restarts every run from new prior draws (device [d][P] when on_device);
 * run i gets seed + i. */
smc_status smc_batch_reset(smc_batch* b, const double* const* theta0s, int theta0_on_device, uint64_t seed);
/* Sums over runs of M-phase particle x observation evaluations and Metropolis
 * iterations, and batched cycles so far (host outputs, nullable). */
smc_status smc_batch_totals(smc_batch* b, double* evals, int64_t* metropolis_steps, int* cycles);
/* Run i's context, for smc_log_ml, smc_moments, smc_get_particles,
 * smc_run_totals (owned by the batch). */
smc_ctx* smc_batch_member(smc_batch* b, int i);
int smc_batch_tile(const smc_batch* b);
const char* smc_batch_last_error(const smc_batch* b);
void smc_batch_free(smc_batch* b);

/* ---------------------------------------------------------------------------
 * Stateless entry points on caller-owned device memory (for tests, autograd
 * and custom drivers).  All enqueue on `stream`; temporaries they need are
 * allocated stream-ordered (cudaMallocAsync) and released before return.
 * ------------------------------------------------------------------------- */

/* Log likelihood log p(y_1:T | theta) of Section 5.1 (four evaluation steps)
 * for P particles.  obs: device observations, float[T] for EGARCH with
 * SMC_FP32, double[T] for EGARCH with SMC_FP64, or double[T][W] records
 * [x_1..x_p, y, 0...] with W = smc_linreg_width(p) for LINREG; 16-byte
 * aligned.  theta: device [d][P].  Outputs (device, nullable except ll):
 * ll[P], lp[P] (log prior), state[K+1][P] (v_kT, eps_T). */
smc_status smc_loglik(const smc_model* m, int precision, const void* obs, int T,
                      const double* theta, int P, double* ll, double* lp, double* state,
                      void* stream);
int smc_linreg_width(int p);

/* One random-walk Metropolis iteration (Section 3.3) on device particles in
 * place: proposal theta + L z with z from Philox4x64-10 at counter
 * (particle, iter, cycle, 1 << 32 | block), acceptance against
 * lp + phi * ll with log u from counter (particle, iter, cycle, 2 << 32).
 * L: device [d][d] lower triangular, row-major.  accepted (host, nullable)
 * receives the number of accepted proposals (synchronises). */
smc_status smc_mutate_rw(const smc_model* m, int precision, const void* obs, int T,
                         double* theta, double* ll, double* lp, double* state, int P,
                         const double* L, double phi, uint64_t seed, uint64_t cycle,
                         uint64_t iter, uint64_t* accepted, void* stream);

/* Log likelihood and its gradient with respect to the (free) transformed
 * parameters theta, by a hand-written adjoint (reverse-mode) sweep through the
 * EGARCH recursion of Section 5.1 with checkpoints of the state every 32 (FP32)
 * or 16 (FP64) observations; for LINREG the closed form sum_t (y_t - x_t'b) x_t
 * / sigma^2.  Layouts as smc_loglik; grad: device [d][P].  Checkpoint scratch
 * is allocated stream-ordered (about (K+1) T P / 32 values). */
smc_status smc_loglik_grad(const smc_model* m, int precision, const void* obs, int T,
                           const double* theta, int P, double* ll, double* grad, double* state,
                           void* stream);

/* One independent Gaussian Metropolis iteration (Section 3.3's alternative
 * sampler) on device particles in place: proposal mean + L z with z as in
 * smc_mutate_rw, accepted with log u < [lp + phi l](theta*) - [lp + phi l](theta)
 * + log q(theta) - log q(theta*), q = N(mean, L L'); log q(theta) is
 * -|L^{-1}(theta - mean)|^2 / 2 by forward substitution in FP64, a zero pivot of
 * L contributing nothing.  mean: device [d]; other arguments as smc_mutate_rw.
 * The paper has no kernel for it; the acceptance rule is the standard
 * Metropolis-Hastings ratio for an independence proposal. */
smc_status smc_mutate_indep(const smc_model* m, int precision, const void* obs, int T,
                            double* theta, double* ll, double* lp, double* state, int P,
                            const double* mean, const double* L, double phi, uint64_t seed,
                            uint64_t cycle, uint64_t iter, uint64_t* accepted, void* stream);

/* One MALA iteration on device particles in place (an alternative Metropolis
 * update in the sense of Section 3.3): theta* = theta + (1/2) L L' g + L z,
 * g = grad log prior + phi grad (stored gradient of the log likelihood, device
 * [d][P], updated on acceptance), z as in smc_mutate_rw; accepted with
 * log u < [lp + phi l](theta*) - [lp + phi l](theta) + log q(theta | theta*)
 * - log q(theta* | theta).  accepted (host, nullable) synchronises. */
smc_status smc_mutate_mala(const smc_model* m, int precision, const void* obs, int T, double* theta,
                           double* ll, double* lp, double* grad, double* state, int P, const double* L,
                           double phi, uint64_t seed, uint64_t cycle, uint64_t iter, uint64_t* accepted,
                           void* stream);

/* Pooled mean and covariance V of theta (device [d][P]) and the lower
 * Cholesky factor of (h_tenths / 10)^2 V (Section 3.3, Sigma = h^2 V); a
 * non-positive pivot zeroes its column.  Outputs (device, nullable): mean[d],
 * cov[d][d], L[d][d]. */
smc_status smc_cov_chol(const double* theta, int d, int P, int h_tenths, double* mean,
                        double* cov, double* L, void* stream);

/* Power tempering C phase: the increment dphi in (0, 1 - phi] at which the
 * pooled RSS of weights exp(dphi * ll) first falls below d1, by `passes`
 * k-ary passes of 32 candidates (evenly spaced over the current bracket, the
 * bracket narrowing to the first candidate below d1 and its predecessor);
 * 1 - phi if RSS(1 - phi) >= d1.  The candidate weights are FP32
 * exponentials whose sums are exact 64-bit fixed-point totals, so the result
 * does not depend on the grid; RSS is compared with d1 to about 1e-7.  One
 * cooperative launch.  ll: device [P] (NaN counts as -inf).  Host outputs:
 * dphi, rss (FP64 RSS at dphi).  Synchronises. */
smc_status smc_power_search(const double* ll, int P, double phi, double d1, int passes,
                            double* dphi, double* rss, void* stream);

/* S phase within each of J groups of N (Section 3.3): residual
 * (SMC_RESIDUAL), multinomial, stratified or systematic resampling (the last
 * two: slot k takes the particle whose inclusive prefix of q first exceeds
 * floor((k Q + U_k) / N), U_k = mulhi64(x, Q), with one Philox draw per group
 * (systematic, draw index 0) or per slot (stratified)) from weights w (device [J*N],
 * non-negative, any scale per group).  Integer fixed point: q_n =
 * floor(2^32 w_n / max w), counts floor(N q_n / Q), residual draws by
 * upper_bound on the integer residual prefix with mulhi64(x, R), x from
 * Philox4x64-10 at counter (group, draw, cycle, 3 << 32).  idx: device
 * [J*N] int32, group-local source index of each output slot, in particle
 * order.  Returns SMC_EDEGENERATE if a group's weights are all zero. */
smc_status smc_resample(const double* w, int J, int N, int resampler, uint64_t seed,
                        uint64_t cycle, int32_t* idx, void* stream);

/* The S phase as a run takes it, from log weights (Section 3.3 for the
 * resampling, Section 4.2 for the group weight): logw is device [J*N]
 * (-inf for a particle of weight zero), w_n = exp(logw_n - max_n logw_n),
 * then exactly smc_resample on those weights.  The quantised weights
 * floor(2^32 w_n) are those of the FP64 exponential; the kernel evaluates
 * them in 64-bit fixed point and falls back to the FP64 exponential only
 * where 2^32 w_n lies within 2^-18 of an integer.  lwbar: host [J] or NULL,
 * receives log wbar_j = max + log(sum_n w_n / N) with the sums formed
 * exactly in fixed point.  Returns SMC_EDEGENERATE if every log weight of a
 * group is -inf (its slots then keep their own particles).  Synchronises. */
smc_status smc_resample_logw(const double* logw, int J, int N, int resampler, uint64_t seed,
                             uint64_t cycle, int32_t* idx, double* lwbar, void* stream);

/* Grand mean, s.d., NSE and RNE (Section 2.3) of each of nf functions
 * g (device [nf][J*N], group-major columns).  out: host [nf][4]. */
smc_status smc_group_moments(const double* g, int nf, int J, int N, double* out, void* stream);

/* The same computation as smc_cov_chol for callers that cannot allocate
 * device memory while they run (a framework that reserves the device memory
 * budget up front, or a latency-bound loop that must not wait on the memory
 * pool).  The paper has no counterpart: this is a deployment variant.  Its
 * partial-sum scratch is a fixed array inside the library (about 2.3 MB per
 * device that uses it, held until the process exits), so it calls no
 * allocator.  It splits the particles over the same blocks as smc_cov_chol
 * (at most 512 blocks: identical results on any device with up to 256 SMs,
 * equal within FP rounding of the sums beyond).  Limits: 1 <= d <= SMC_MAX_D,
 * P >= 2; other sizes return SMC_EINVAL.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point after a
 * cudaDeviceReset in the same process.  All calls on a device share the array:
 * calls whose kernels overlap on the GPU (unordered streams) race on it.
 * Every partial sum read in a call is written earlier in the same call and
 * the reduction's counter (the array's last word) is back at zero when a call
 * ends, so no clearing is needed.  Arguments, outputs and errors as
 * smc_cov_chol. */
smc_status smc_cov_chol_noalloc(const double* theta, int d, int P, int h_tenths, double* mean,
                                double* cov, double* L, void* stream);

/* log wbar, its NSE (ML_se) from per-group log products a (device [J]). */
smc_status smc_ml_from_groups(const double* a, int J, double* log_ml, double* nse, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
