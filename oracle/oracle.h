/*
 * Plain FP64 CPU oracle for the adaptive sequential posterior simulator of
 * Durham & Geweke, "Adaptive Sequential Posterior Simulators for Massively
 * Parallel Computing Environments" (2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * or run it.  It shares no source with the CUDA library: it has its own Philox,
 * its own model code, its own C/S/M phases and its own estimators.  Everything is
 * double precision, single threaded unless a thread count is passed, and written
 * in the order and notation of the paper so that it can be read against it.
 *
 * Parity notes per function are in the .c files.  Pinning (what each function is
 * checked against other than itself) lives in tests/test_oracle_*.py.
 * Parity unpinned: the full EGARCH K>=2 SMC run has no closed form; it is pinned
 * only statistically (agreement within combined NSE across configurations).
 */
#ifndef SMC_ORACLE_H
#define SMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------- */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* M-phase proposal normals z[0..d) of particle p at (cycle, iter): Box-Muller on
 * the four 53-bit uniforms of each Philox block (tag OR_TAG_M_NORMAL, block b). */
void or_philox_normals(uint64_t seed, uint64_t p, uint64_t iter, uint64_t cycle,
                       int d, double *z);
/* log u of the Metropolis-Hastings uniform of particle p at (cycle, iter). */
double or_philox_log_uniform(uint64_t seed, uint64_t p, uint64_t iter, uint64_t cycle);

/* Counter-map tags shared by convention (not code) with the CUDA path. */
#define OR_TAG_M_NORMAL  1u   /* Gaussian proposal normals (M phase)          */
#define OR_TAG_M_UNIFORM 2u   /* Metropolis-Hastings uniform (M phase)        */
#define OR_TAG_S_RESID   3u   /* residual / multinomial draws (S phase)       */
#define OR_TAG_C_PIT     4u   /* PIT auxiliary draw Y_s (C phase, Section 4.1) */
#define OR_TAG_PRIOR     5u   /* prior draws (Table 1)                         */

/* ---- model description ---------------------------------------------------- */
enum { OR_EGARCH = 0, OR_LINREG = 1 };

typedef struct {
    int model;                 /* OR_EGARCH | OR_LINREG                          */
    int K, I, gamma;           /* EGARCH: factors, mixture comps, leverage term  */
    int p;                     /* LINREG: regressors                             */
    double sigma;              /* LINREG: known disturbance s.d.                 */
    int d_full;                /* full parameter count of the model              */
    int d;                     /* parameters carried by particles (free)         */
    const int *free_idx;       /* [d] position of each free parameter in full    */
    const double *theta_fixed; /* [d_full] values of the non-free parameters     */
    const double *prior_mean;  /* [d] Gaussian prior on each free parameter      */
    const double *prior_sd;    /* [d]                                            */
    const double *prior_lo;    /* [d] truncation from below (-inf: none)         */
    int eps0_zero;             /* 0: v_k1 = 0 (default); 1: eps_0 = 0 reading    */
} or_model;

/* EGARCH parameter count of Table 1 for the chosen shape. */
int or_egarch_dim(int K, int I, int gamma);
/* Table 1 prior over the full EGARCH vector (mean, s.d., lower truncation). */
void or_egarch_prior_table1(int K, int I, int gamma, double *mean, double *sd, double *lo);

/* EGARCH model parameters after Table 1 transforms and (EGARCH_tran1/2). */
typedef struct {
    double mu_y, sigma_y;
    double alpha[8], beta[8], gamma[8];
    double p[8], mu[8], sig[8];
} or_egarch_par;
void or_egarch_transform(int K, int I, int gamma, const double *theta_full, or_egarch_par *par);

/* Full parameter vector from the free ones (fixed values fill the rest). */
void or_full_theta(const or_model *m, const double *theta, double *full);

/* Log prior density kernel over free parameters; -inf outside the support. */
double or_logprior(const or_model *m, const double *theta);

/* Log likelihood log p(y_{1:T} | theta) for one particle (theta = free params).
 * state_out (nullable): EGARCH end state [K+1] = (v_{1T}..v_{KT}, eps_T).      */
double or_loglik(const or_model *m, const double *y, const double *X, int T,
                 const double *theta, double *state_out);
/* Continue an EGARCH recursion from a saved end state at t0 (t0 >= 1) through
 * observation t1 (1-based inclusive); returns the sum of log densities and
 * updates state in place.  With t0 == 0 it is the plain likelihood.            */
double or_loglik_range(const or_model *m, const double *y, const double *X,
                       int t0, int t1, const double *theta, double *state);
/* Per-observation log densities l_t, t = 1..T, into lt[T]. */
void or_loglik_terms(const or_model *m, const double *y, const double *X, int T,
                     const double *theta, double *lt);
/* Gradient of log p(y_{1:T}|theta) w.r.t. the free parameters, by forward-mode
 * (dual-number) differentiation of the same recursion.  Returns the loglik.    */
double or_loglik_grad(const or_model *m, const double *y, const double *X, int T,
                      const double *theta, double *grad);
/* Gradient of the log prior kernel. */
void or_logprior_grad(const or_model *m, const double *theta, double *grad);

/* Test functions g1, g2, g3 of Section 5.2 at the end of the recursion. */
void or_egarch_testfn(const or_model *m, const double *theta, const double *state,
                      double g[3]);

/* Batch helpers over P particles, theta row-major [P][d]. */
void or_loglik_batch(const or_model *m, const double *y, const double *X, int T,
                     const double *theta, int P, double *loglik, double *state,
                     int nthreads);
void or_logprior_batch(const or_model *m, const double *theta, int P, double *lp);

/* ---- estimators (Section 2.3, Section 4.2) --------------------------------- */
/* Grand mean, NSE and RNE of g over J groups of N (g[J*N], group-major).      */
void or_moment(const double *g, int J, int N, double *mean, double *sd,
               double *nse, double *rne);
/* Effective sample size of weights given as log weights over n particles.     */
double or_ess_log(const double *logw, int n);
/* Log marginal likelihood from per-group log products a_j = sum_l log wbar_j. */
void or_log_ml(const double *a, int J, double *log_ml, double *nse_log);

/* ---- S phase (Section 3.3 "Resampling method") ------------------------------ */
/* Residual (resid=1) or multinomial (resid=0) resampling within each of J
 * groups of N particles from weights w[J*N] (need not be normalised).  idx[J*N]
 * receives the source particle index (group-local) for each output slot.
 * The quantisation and draws follow the fixed-point reading documented in the
 * .c file.  Returns 0, or -1 if a group has zero total weight.                */
int or_resample(const double *w, int J, int N, int resid, uint64_t seed,
                uint64_t cycle, int32_t *idx);

/* Resampling by scheme: 0 residual, 1 multinomial, 2 stratified, 3 systematic
 * (the last two are the paper's experimental alternatives). */
int or_resample_scheme(const double *w, int J, int N, int scheme, uint64_t seed,
                       uint64_t cycle, int32_t *idx);

/* ---- prior draws (Table 1; truncation by rejection) ------------------------ */
/* theta[P][d] (free parameters): component i of particle n at attempt a is
 * normal i % 4 of the Philox block (n, a, 0, OR_TAG_PRIOR << 32 | i / 4).     */
void or_draw_prior(const or_model *m, uint64_t seed, int P, double *theta);

/* ---- probability integral transform (Section 4.1) -------------------------- */
/* Simulated standardized shock of Y_s ~ p(Y_s | y_{1:s-1}, theta) for particle
 * `particle` (Philox counter (particle, s, 0, OR_TAG_C_PIT << 32)), and the
 * observed one e_s (EGARCH: from the state after the step through y_s).
 * Y_s <= y_s exactly when the simulated shock is <= e_s.                      */
double or_pit_shock(const or_model *m, const double *theta, uint64_t seed,
                    uint64_t particle, int s);
double or_obs_shock(const or_model *m, const double *y, const double *X, int s,
                    const double *theta, const double *state_after);

/* ---- covariance & Cholesky (Section 3.3 "Metropolis steps") ---------------- */
void or_mean_cov(const double *theta, int P, int d, double *mean, double *cov);
int or_cholesky(const double *A, int d, double *L); /* lower, row-major */

/* ---- M phase ---------------------------------------------------------------- */
/* One Gaussian random-walk Metropolis step on every particle (in place).
 * Proposal theta' = theta + L z, z ~ N(0, I) from Philox; L = chol(h^2 V).
 * Target: logprior + phi * loglik.  accept[P] (nullable) gets 0/1.
 * Returns the number of accepted proposals.                                  */
long or_mutate_rw(const or_model *m, const double *y, const double *X, int T,
                  double *theta, double *loglik, double *logprior, double *state,
                  int P, const double *L, double phi, uint64_t seed,
                  uint64_t cycle, uint64_t iter, int *accept, int nthreads);
/* One MALA step: theta' = theta + (1/2) Sigma grad + L z with Sigma = L L^T.
 * grad[P*d] holds the gradient of the log likelihood at the current theta and
 * is updated on acceptance.                                                  */
long or_mutate_mala(const or_model *m, const double *y, const double *X, int T,
                    double *theta, double *loglik, double *logprior, double *grad,
                    double *state, int P, const double *L, double phi,
                    uint64_t seed, uint64_t cycle, uint64_t iter, int *accept,
                    int nthreads);

/* One independent Gaussian Metropolis step (Section 3.3's alternative
 * sampler): theta' = mbar + L z with q = N(mbar, L L^T) the same for every
 * particle; acceptance includes log q(theta) - log q(theta').  A zero pivot of
 * L contributes nothing to log q (the oracle's singular-factor rule).         */
long or_mutate_indep(const or_model *m, const double *y, const double *X, int T,
                     double *theta, double *loglik, double *logprior, double *state,
                     int P, const double *mbar, const double *L, double phi,
                     uint64_t seed, uint64_t cycle, uint64_t iter, int *accept,
                     int nthreads);

/* ---- C phase ---------------------------------------------------------------- */
/* Power tempering: find dphi in (0, 1-phi] with RSS(dphi) = D1 by bisection
 * (RSS(1-phi) >= D1 gives 1-phi).  Returns dphi; rss_out gets RSS(dphi).     */
double or_power_search(const double *loglik, int P, double phi, double d1,
                       int iters, double *rss_out);

/* ---- full run (Algorithm 2 with the Section 3.3 specifics) ------------------ */
typedef struct {
    int J, N;
    int tempering;      /* 0 = data (paper), 1 = power                          */
    int mutation;       /* 0 = random walk, 1 = MALA, 2 = independent Gaussian
                           (Sigma = V, the pooled variance; mean = pooled mean;
                           no replay or recording)                           */
    int resid;          /* 1 residual, 0 multinomial, 2 stratified, 3 systematic */
    double d1, d2;
    int stop_rule;      /* 0 deterministic, 1 RNE                               */
    int rbar, kappa, rmax;
    double e1, e2;
    int h0_tenths, hmin_tenths, hmax_tenths; /* step size in tenths            */
    double acc_target;
    int h_reset_each_cycle;
    const int *force_dates; int n_force; /* data tempering dates of interest   */
    int bisect_iters;
    uint64_t seed;
    int max_cycles;
    int nthreads;
    /* Algorithm 3 (hybrid).  Recording (rec_L non-NULL, capacity rec_L_cap
     * iterations): the Cholesky factor of every Metropolis iteration's
     * Sigma_lr is stored, d*d each, in order.  Replay (replay = 1): cycle l ends
     * at design_x[l] (t_l in data tempering, phi_l in power tempering), runs
     * design_R[l] iterations with the stored factors design_L in order; no
     * adaptation.  n_design cycles. */
    int replay;
    int n_design;
    const double *design_x;
    const int *design_R;
    const double *design_L;
    double *rec_L;
    int rec_L_cap;
    /* Section 4.1 (data tempering only).  burnin b > 0: a cycle ends at t = b
     * and the log score log p(y_{b+1:T} | y_{1:b}) is the group-product
     * estimator over the cycles after b.  pit_out[T] (nullable): at each s the
     * weighted fraction of particles whose simulated Y_s is <= y_s, with the
     * weights w(s-1) of the C phase. */
    int burnin;
    double *pit_out;
} or_run_cfg;

typedef struct {
    int cycles;
    long metropolis_steps;
    double particle_obs_evals;    /* M phase sum over r of P * t_l             */
    double log_ml, log_ml_nse, log_ml_tilde;
    int h_final_tenths;
    int status;                   /* 0 ok; <0 error                             */
    double log_score, log_score_nse;  /* NaN without a burn-in               */
} or_run_out;

/* Runs the simulator from prior draws theta0[P][d] to the full sample.  On
 * return theta/loglik/logprior/state hold the final particles (caller-owned,
 * sized P*d, P, P, P*(K+1)), a_out[J] the per-group log ML accumulators, and
 * per-cycle records (nullable, sized max_cycles): t_l, phi_l, R_l, rss_l.    */
int or_smc_run(const or_model *m, const double *y, const double *X, int T,
               const or_run_cfg *cfg, const double *theta0,
               double *theta, double *loglik, double *logprior, double *state,
               double *a_out, int *t_rec, double *phi_rec, int *r_rec,
               double *rss_rec, or_run_out *out);

#ifdef __cplusplus
}
#endif
#endif
