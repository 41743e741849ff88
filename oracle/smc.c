/*
 * Oracle for the sequential posterior simulator: estimators, C, S and M phases,
 * and the full adaptive run.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Passages followed:
 *   - grand mean, NSE, RNE: (garnd_approx), (vhat), (NSE_def) and the RNE
 *     definition of Section 2.3
 *   - Algorithm 1 / Algorithm 2 structure (C, S, M phases per cycle)
 *   - Section 3.3: ESS/RSS C-phase termination, residual resampling, Gaussian
 *     random-walk Metropolis with Sigma = h^2 V and the h adaptation rule, the
 *     deterministic and RNE-based M-phase stopping rules
 *   - Section 4.2: wbar_j, wbar, wtilde and the working NSE (ML_se)
 * Readings where the paper is silent (each mirrored by the CUDA path):
 *   - ESS, the covariance V and the acceptance rate are pooled over all J*N.
 *   - h is held in tenths, starts at h0 once per run, is updated after every
 *     Metropolis iteration (+1 if acceptance > target, else -1, clamped).
 *   - power tempering (an addition to the paper's data tempering): target
 *     p(theta) p(y|theta)^phi; the increment dphi is found by bisection so that
 *     RSS just falls below D1; if RSS(1-phi) >= D1 the increment is 1-phi.
 *   - residual resampling in integer fixed point: q_n = floor(2^32 w_n/max w),
 *     count_n = floor(N q_n / Q), residuals r_n = N q_n - Q count_n, and the
 *     N - sum count residual draws pick upper_bound(prefix r, mulhi64(x, R)) with
 *     x from Philox.  Multinomial is the same with all counts zero.  With 32
 *     fractional bits the residual total R = Q (N - sum count) stays below 2^64
 *     for N up to 2^15 (Q <= N 2^32); a particle whose weight is below 2^-32 of
 *     the group maximum is never selected, which moves at most N 2^-32 of the
 *     selection probability.
 *   - RNE stopping rule: arithmetic mean of the RNE of the test functions after
 *     each iteration; E1 normally, E2 at dates of interest and at the end of the
 *     sample; at most Rmax iterations.
 *   - Random numbers: Philox4x64-10 with key (seed, 0) and counter
 *     (particle, iteration, cycle, tag << 32 | block); uniforms
 *     ((x >> 11) + 0.5) 2^-53; normals by Box-Muller on consecutive pairs.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_POW_M53 (1.0 / 9007199254740992.0)

static double u53(uint64_t x) { return ((double)(x >> 11) + 0.5) * TWO_POW_M53; }

/* Proposal normals z[0..d) for one particle. */
void or_philox_normals(uint64_t seed, uint64_t p, uint64_t iter, uint64_t cycle,
                           int d, double *z)
{
    const uint64_t key[2] = {seed, 0};
    for (int b = 0; 4 * b < d; ++b) {
        uint64_t ctr[4] = {p, iter, cycle, ((uint64_t)OR_TAG_M_NORMAL << 32) | (uint64_t)b};
        uint64_t out[4];
        or_philox4x64(ctr, key, out);
        for (int pair = 0; pair < 2; ++pair) {
            double ua = u53(out[2 * pair]), ub = u53(out[2 * pair + 1]);
            double rho = sqrt(-2.0 * log(ua));
            double ang = 2.0 * M_PI * ub;
            int n = 4 * b + 2 * pair;
            if (n < d) z[n] = rho * cos(ang);
            if (n + 1 < d) z[n + 1] = rho * sin(ang);
        }
    }
}

double or_philox_log_uniform(uint64_t seed, uint64_t p, uint64_t iter, uint64_t cycle)
{
    const uint64_t key[2] = {seed, 0};
    uint64_t ctr[4] = {p, iter, cycle, (uint64_t)OR_TAG_M_UNIFORM << 32};
    uint64_t out[4];
    or_philox4x64(ctr, key, out);
    return log(u53(out[0]));
}

/* ------------------------------ prior draws ------------------------------- */
/* Table 1 priors: theta_i = m_i + s_i z_i, z_i standard normal; a component
 * with a finite lower bound (theta_8i >= -3) is redrawn until it is inside
 * (truncation by rejection).  The draw of component i at attempt a is normal
 * i % 4 of the Philox block at counter (particle, a, 0, tag 5 << 32 | i / 4):
 * Box-Muller on the uniform pairs (0,1) -> normals 0 (cos), 1 (sin) and
 * (2,3) -> normals 2, 3.  After 64 rejected attempts the bound itself is used. */
void or_draw_prior(const or_model *m, uint64_t seed, int P, double *theta)
{
    const uint64_t key[2] = {seed, 0};
    const int d = m->d;
    for (int n = 0; n < P; ++n)
        for (int i = 0; i < d; ++i) {
            double x = m->prior_lo[i];
            for (int a = 0; a < 64; ++a) {
                uint64_t ctr[4] = {(uint64_t)n, (uint64_t)a, 0, ((uint64_t)OR_TAG_PRIOR << 32) | (uint64_t)(i / 4)};
                uint64_t out[4];
                or_philox4x64(ctr, key, out);
                const int pair = (i % 4) / 2;
                double rho = sqrt(-2.0 * log(u53(out[2 * pair])));
                double ang = 2.0 * M_PI * u53(out[2 * pair + 1]);
                double z = (i % 2 == 0) ? rho * cos(ang) : rho * sin(ang);
                double v = m->prior_mean[i] + m->prior_sd[i] * z;
                if (v >= m->prior_lo[i]) { x = v; break; }
            }
            theta[(size_t)n * d + i] = x;
        }
}

/* ------------------------ probability integral transform ------------------ */
/* Section 4.1: Y_s ~ p(Y_s | y_{1:s-1}, theta) is location + scale * e with e the
 * standardized shock (EGARCH: location mu_Y, scale h_s; LINREG: x_s'beta and
 * sigma), so I[Y_s <= y_s] = I[e <= e_s].  The simulated e takes mixture
 * component i when the uniform u_c falls in [p_1 + .. + p_{i-1}, p_1 + .. + p_i),
 * then mu_i + sigma_i z (LINREG: z), z Box-Muller from the next two uniforms;
 * all three come from the Philox block at counter (particle, s, 0, tag 4). */
double or_pit_shock(const or_model *m, const double *theta, uint64_t seed,
                    uint64_t particle, int s)
{
    const uint64_t key[2] = {seed, 0};
    uint64_t ctr[4] = {particle, (uint64_t)s, 0, (uint64_t)OR_TAG_C_PIT << 32};
    uint64_t out[4];
    or_philox4x64(ctr, key, out);
    double uc = u53(out[0]);
    double z = sqrt(-2.0 * log(u53(out[1]))) * cos(2.0 * M_PI * u53(out[2]));
    if (m->model == OR_LINREG) return z;
    double full[64];
    or_full_theta(m, theta, full);
    or_egarch_par q;
    or_egarch_transform(m->K, m->I, m->gamma, full, &q);
    int comp = m->I - 1;
    double cum = 0.0;
    for (int i = 0; i < m->I; ++i) {
        cum += q.p[i];
        if (uc < cum) { comp = i; break; }
    }
    return q.mu[comp] + q.sig[comp] * z;
}

/* Observed standardized shock e_s: EGARCH reads eps_s from the state after the
 * step through y_s; LINREG computes (y_s - x_s'beta) / sigma. */
double or_obs_shock(const or_model *m, const double *y, const double *X, int s,
                    const double *theta, const double *state_after)
{
    if (m->model == OR_EGARCH) return state_after[m->K];
    double full[64];
    or_full_theta(m, theta, full);
    double mean = 0.0;
    for (int i = 0; i < m->p; ++i) mean += X[(size_t)(s - 1) * m->p + i] * full[i];
    return (y[s - 1] - mean) / m->sigma;
}

/* ------------------------------ estimators -------------------------------- */
void or_moment(const double *g, int J, int N, double *mean, double *sd,
               double *nse, double *rne)
{
    double *gj = malloc(sizeof(double) * (size_t)J);
    double gbar = 0.0;
    for (int j = 0; j < J; ++j) {
        double s = 0.0;
        for (int n = 0; n < N; ++n) s += g[(size_t)j * N + n];
        gj[j] = s / N;                                    /* gbar_j^N */
        gbar += gj[j];
    }
    gbar /= J;                                            /* (garnd_approx) */
    double between = 0.0;
    for (int j = 0; j < J; ++j) between += (gj[j] - gbar) * (gj[j] - gbar);
    double total = 0.0;
    for (size_t i = 0; i < (size_t)J * N; ++i) total += (g[i] - gbar) * (g[i] - gbar);
    double var_hat = total / ((double)N * J - 1.0);       /* var-hat of g */
    double v_hat = (double)N / (J - 1.0) * between;        /* (vhat) */
    *mean = gbar;
    *sd = sqrt(var_hat);
    *nse = sqrt(between / ((double)J * (J - 1.0)));       /* (NSE_def) */
    *rne = v_hat > 0.0 ? var_hat / v_hat : INFINITY;
    free(gj);
}

double or_ess_log(const double *logw, int n)
{
    double m = -INFINITY;
    for (int i = 0; i < n; ++i) if (logw[i] > m) m = logw[i];
    if (m == -INFINITY) return 0.0;
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = exp(logw[i] - m);
        s1 += w;
        s2 += w * w;
    }
    return s1 * s1 / s2;
}

void or_log_ml(const double *a, int J, double *log_ml, double *nse_log)
{
    double amax = -INFINITY;
    for (int j = 0; j < J; ++j) if (a[j] > amax) amax = a[j];
    double rbar = 0.0;
    for (int j = 0; j < J; ++j) rbar += exp(a[j] - amax);
    rbar /= J;                                  /* wbar / e^{amax} */
    double ss = 0.0;
    for (int j = 0; j < J; ++j) {
        double r = exp(a[j] - amax);
        ss += (r - rbar) * (r - rbar);
    }
    *log_ml = amax + log(rbar);                 /* log wbar^(J,N) */
    *nse_log = sqrt(ss / ((double)J * (J - 1.0))) / rbar;  /* (ML_se) */
}

static double logsumexp(const double *x, int n)
{
    double m = -INFINITY;
    for (int i = 0; i < n; ++i) if (x[i] > m) m = x[i];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(x[i] - m);
    return m + log(s);
}

/* ------------------------------- S phase ---------------------------------- */
static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* Stratified (scheme 2) and systematic (scheme 3) resampling, Section 3.3's
 * experimental alternatives, in the same fixed point: with q_n and Q as for
 * residual resampling, output slot k takes the particle whose inclusive prefix
 * of q first exceeds pos_k = floor((k Q + U_k) / N), U_k = mulhi64(x_k, Q);
 * systematic uses one draw x_0 for all k (counter (group, 0, cycle, 3<<32)),
 * stratified one draw per slot (counter (group, k, cycle, 3<<32)). */
static void resample_strat_sys(const uint64_t *q, uint64_t Q, int N, int systematic, uint64_t seed,
                               uint64_t group, uint64_t cycle, int32_t *idx)
{
    const uint64_t key[2] = {seed, 0};
    uint64_t U0 = 0;
    if (systematic) {
        uint64_t ctr[4] = {group, 0, cycle, (uint64_t)OR_TAG_S_RESID << 32}, out[4];
        or_philox4x64(ctr, key, out);
        U0 = mulhi64(out[0], Q);
    }
    for (int k = 0; k < N; ++k) {
        uint64_t U = U0;
        if (!systematic) {
            uint64_t ctr[4] = {group, (uint64_t)k, cycle, (uint64_t)OR_TAG_S_RESID << 32}, out[4];
            or_philox4x64(ctr, key, out);
            U = mulhi64(out[0], Q);
        }
        const uint64_t pos = ((uint64_t)k * Q + U) / (uint64_t)N;
        uint64_t acc = 0;
        int pick = N - 1;
        for (int n = 0; n < N; ++n) {
            acc += q[n];
            if (acc > pos) { pick = n; break; }
        }
        idx[k] = pick;
    }
}

int or_resample_scheme(const double *w, int J, int N, int scheme, uint64_t seed, uint64_t cycle,
                       int32_t *idx)
{
    if (scheme <= 1) return or_resample(w, J, N, scheme == 1 ? 0 : 1, seed, cycle, idx);
    uint64_t *q = malloc(sizeof(uint64_t) * (size_t)N);
    int status = 0;
    for (int j = 0; j < J; ++j) {
        const double *wj = w + (size_t)j * N;
        double wmax = 0.0;
        for (int n = 0; n < N; ++n) if (wj[n] > wmax) wmax = wj[n];
        if (!(wmax > 0.0) || !isfinite(wmax)) { status = -1; continue; }
        uint64_t Q = 0;
        for (int n = 0; n < N; ++n) {
            double wn = wj[n] > 0.0 ? wj[n] / wmax : 0.0;
            q[n] = (uint64_t)floor(ldexp(wn, 32));
            Q += q[n];
        }
        resample_strat_sys(q, Q, N, scheme == 3, seed, (uint64_t)j, cycle, idx + (size_t)j * N);
    }
    free(q);
    return status;
}

int or_resample(const double *w, int J, int N, int resid, uint64_t seed,
                uint64_t cycle, int32_t *idx)
{
    uint64_t *q = malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *cnt = malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *r = malloc(sizeof(uint64_t) * (size_t)N);
    int status = 0;
    const uint64_t key[2] = {seed, 0};
    for (int j = 0; j < J; ++j) {
        const double *wj = w + (size_t)j * N;
        double wmax = 0.0;
        for (int n = 0; n < N; ++n) if (wj[n] > wmax) wmax = wj[n];
        if (!(wmax > 0.0) || !isfinite(wmax)) { status = -1; continue; }
        uint64_t Q = 0;
        for (int n = 0; n < N; ++n) {
            double wn = wj[n] > 0.0 ? wj[n] / wmax : 0.0;
            q[n] = (uint64_t)floor(ldexp(wn, 32));
            Q += q[n];
        }
        uint64_t placed = 0, R = 0;
        for (int n = 0; n < N; ++n) {
            if (resid) {
                cnt[n] = ((uint64_t)N * q[n]) / Q;               /* floor(N w~_n) */
                r[n] = (uint64_t)N * q[n] - Q * cnt[n];
            } else {
                cnt[n] = 0;
                r[n] = q[n];
            }
            placed += cnt[n];
            R += r[n];
        }
        uint64_t M = (uint64_t)N - placed;
        for (uint64_t mdraw = 0; mdraw < M; ++mdraw) {
            uint64_t ctr[4] = {(uint64_t)j, mdraw, cycle, (uint64_t)OR_TAG_S_RESID << 32};
            uint64_t out[4];
            or_philox4x64(ctr, key, out);
            uint64_t u = mulhi64(out[0], R);           /* uniform on [0, R) */
            /* upper_bound: first n with prefix_r(n) > u */
            uint64_t acc = 0;
            int pick = N - 1;
            for (int n = 0; n < N; ++n) {
                acc += r[n];
                if (acc > u) { pick = n; break; }
            }
            cnt[pick] += 1;
        }
        int32_t *ij = idx + (size_t)j * N;
        int slot = 0;
        for (int n = 0; n < N; ++n)
            for (uint64_t c = 0; c < cnt[n]; ++c) ij[slot++] = n;
    }
    free(q); free(cnt); free(r);
    return status;
}

/* -------------------------- covariance, Cholesky -------------------------- */
void or_mean_cov(const double *theta, int P, int d, double *mean, double *cov)
{
    for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int n = 0; n < P; ++n) s += theta[(size_t)n * d + i];
        mean[i] = s / P;
    }
    for (int i = 0; i < d; ++i)
        for (int k = 0; k <= i; ++k) {
            double s = 0.0;
            for (int n = 0; n < P; ++n)
                s += (theta[(size_t)n * d + i] - mean[i]) * (theta[(size_t)n * d + k] - mean[k]);
            cov[i * d + k] = cov[k * d + i] = s / (P - 1.0);
        }
}

/* Lower Cholesky factor; a non-positive pivot zeroes that column (the proposal
 * then does not move along it).  Returns the number of zeroed pivots. */
int or_cholesky(const double *A, int d, double *L)
{
    int zeroed = 0;
    memset(L, 0, sizeof(double) * (size_t)d * d);
    for (int i = 0; i < d; ++i) {
        for (int k = 0; k <= i; ++k) {
            double s = A[i * d + k];
            for (int m = 0; m < k; ++m) s -= L[i * d + m] * L[k * d + m];
            if (i == k) {
                if (s > 0.0) L[i * d + i] = sqrt(s);
                else { L[i * d + i] = 0.0; ++zeroed; }
            } else {
                L[i * d + k] = L[k * d + k] > 0.0 ? s / L[k * d + k] : 0.0;
            }
        }
    }
    return zeroed;
}

/* -------------------------------- M phase --------------------------------- */
static double target(double lp, double ll, double phi)
{
    if (lp == -INFINITY) return -INFINITY;
    return phi > 0.0 ? lp + phi * ll : lp;
}

long or_mutate_rw(const or_model *m, const double *y, const double *X, int T,
                  double *theta, double *loglik, double *logprior, double *state,
                  int P, const double *L, double phi, uint64_t seed,
                  uint64_t cycle, uint64_t iter, int *accept, int nthreads)
{
    const int d = m->d;
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 0;
    long total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int n = 0; n < P; ++n) {
        double z[64], prop[64], st[9] = {0};
        double *th = theta + (size_t)n * d;
        or_philox_normals(seed, (uint64_t)n, iter, cycle, d, z);
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int k = 0; k <= i; ++k) s += L[i * d + k] * z[k];
            prop[i] = th[i] + s;                                     /* theta* + L z */
        }
        double lp = or_logprior(m, prop);
        double ll = lp == -INFINITY ? -INFINITY : or_loglik(m, y, X, T, prop, st);
        double log_alpha = target(lp, ll, phi) - target(logprior[n], loglik[n], phi);
        double log_u = or_philox_log_uniform(seed, (uint64_t)n, iter, cycle);
        int acc = log_u < log_alpha;
        if (acc) {
            memcpy(th, prop, sizeof(double) * (size_t)d);
            loglik[n] = ll;
            logprior[n] = lp;
            if (state && ns) for (int k = 0; k < ns; ++k) state[(size_t)n * ns + k] = st[k];
        }
        if (accept) accept[n] = acc;
        total += acc;
    }
    return total;
}

/* Sigma g with Sigma = L L^T. */
static void sigma_mul(const double *L, int d, const double *g, double *out)
{
    double tmp[64];
    for (int k = 0; k < d; ++k) {                 /* tmp = L^T g */
        double s = 0.0;
        for (int i = k; i < d; ++i) s += L[i * d + k] * g[i];
        tmp[k] = s;
    }
    for (int i = 0; i < d; ++i) {                 /* out = L tmp */
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += L[i * d + k] * tmp[k];
        out[i] = s;
    }
}

/* -1/2 |L^{-1} r|^2 (zero pivots contribute nothing). */
static double half_quad_inv(const double *L, int d, const double *r)
{
    double u[64], q = 0.0;
    for (int i = 0; i < d; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= L[i * d + k] * u[k];
        u[i] = L[i * d + i] > 0.0 ? s / L[i * d + i] : 0.0;
        q += u[i] * u[i];
    }
    return -0.5 * q;
}

/* Independent Gaussian sampler (Section 3.3, the alternative to the random
 * walk): proposal theta' = mbar + L z, z ~ N(0, I), the same proposal for every
 * particle's current value; accepted when log u is below
 * [target(theta') - target(theta)] + [log q(theta) - log q(theta')], q the
 * N(mbar, L L^T) density, whose normalising constant cancels.
 * log q(theta') - const = -|z|^2 / 2 because theta' - mbar = L z. */
long or_mutate_indep(const or_model *m, const double *y, const double *X, int T,
                     double *theta, double *loglik, double *logprior, double *state,
                     int P, const double *mbar, const double *L, double phi,
                     uint64_t seed, uint64_t cycle, uint64_t iter, int *accept,
                     int nthreads)
{
    const int d = m->d;
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 0;
    long total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int n = 0; n < P; ++n) {
        double z[64], prop[64], r[64], st[9] = {0};
        double *th = theta + (size_t)n * d;
        or_philox_normals(seed, (uint64_t)n, iter, cycle, d, z);
        double zz = 0.0;
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int k = 0; k <= i; ++k) s += L[i * d + k] * z[k];
            prop[i] = mbar[i] + s;
            zz += z[i] * z[i];
            r[i] = th[i] - mbar[i];
        }
        double lp = or_logprior(m, prop);
        double ll = lp == -INFINITY ? -INFINITY : or_loglik(m, y, X, T, prop, st);
        double lq_cur = half_quad_inv(L, d, r);            /* log q(theta)  + const */
        double lq_prop = -0.5 * zz;                         /* log q(theta') + const */
        double log_alpha = target(lp, ll, phi) - target(logprior[n], loglik[n], phi)
                         + lq_cur - lq_prop;
        double log_u = or_philox_log_uniform(seed, (uint64_t)n, iter, cycle);
        int acc = log_u < log_alpha;
        if (acc) {
            memcpy(th, prop, sizeof(double) * (size_t)d);
            loglik[n] = ll;
            logprior[n] = lp;
            if (state && ns) for (int k = 0; k < ns; ++k) state[(size_t)n * ns + k] = st[k];
        }
        if (accept) accept[n] = acc;
        total += acc;
    }
    return total;
}

long or_mutate_mala(const or_model *m, const double *y, const double *X, int T,
                    double *theta, double *loglik, double *logprior, double *grad,
                    double *state, int P, const double *L, double phi,
                    uint64_t seed, uint64_t cycle, uint64_t iter, int *accept,
                    int nthreads)
{
    const int d = m->d;
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 0;
    long total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int n = 0; n < P; ++n) {
        double z[64], prop[64], g[64], gp[64], sg[64], glp[64], gll[64], st[9] = {0};
        double *th = theta + (size_t)n * d;
        double *gl = grad + (size_t)n * d;
        or_logprior_grad(m, th, glp);
        for (int i = 0; i < d; ++i) g[i] = glp[i] + phi * gl[i];   /* grad log target */
        sigma_mul(L, d, g, sg);
        or_philox_normals(seed, (uint64_t)n, iter, cycle, d, z);
        for (int i = 0; i < d; ++i) {
            double s = 0.0;
            for (int k = 0; k <= i; ++k) s += L[i * d + k] * z[k];
            prop[i] = th[i] + 0.5 * sg[i] + s;
        }
        double lp = or_logprior(m, prop);
        double ll = -INFINITY;
        for (int i = 0; i < d; ++i) gll[i] = 0.0;
        if (lp != -INFINITY) {
            ll = or_loglik_grad(m, y, X, T, prop, gll);
            or_loglik(m, y, X, T, prop, st);
        }
        double log_alpha = -INFINITY;
        if (isfinite(ll) && lp != -INFINITY) {
            or_logprior_grad(m, prop, glp);
            for (int i = 0; i < d; ++i) gp[i] = glp[i] + phi * gll[i];
            double sgp[64], rev[64];
            sigma_mul(L, d, gp, sgp);
            for (int i = 0; i < d; ++i) rev[i] = th[i] - prop[i] - 0.5 * sgp[i];
            double lq_rev = half_quad_inv(L, d, rev);     /* log q(theta | theta') */
            double zz = 0.0;
            for (int i = 0; i < d; ++i) zz += z[i] * z[i];
            double lq_fwd = -0.5 * zz;                     /* log q(theta' | theta) */
            log_alpha = target(lp, ll, phi) - target(logprior[n], loglik[n], phi)
                      + lq_rev - lq_fwd;
        }
        double log_u = or_philox_log_uniform(seed, (uint64_t)n, iter, cycle);
        int acc = log_u < log_alpha;
        if (acc) {
            memcpy(th, prop, sizeof(double) * (size_t)d);
            memcpy(gl, gll, sizeof(double) * (size_t)d);
            loglik[n] = ll;
            logprior[n] = lp;
            if (state && ns) for (int k = 0; k < ns; ++k) state[(size_t)n * ns + k] = st[k];
        }
        if (accept) accept[n] = acc;
        total += acc;
    }
    return total;
}

/* -------------------------------- C phase --------------------------------- */
static double rss_power(const double *loglik, int P, double llmax, double dphi)
{
    double s1 = 0.0, s2 = 0.0;
    for (int n = 0; n < P; ++n) {
        if (loglik[n] == -INFINITY) continue;
        double w = exp(dphi * (loglik[n] - llmax));
        s1 += w;
        s2 += w * w;
    }
    return s1 * s1 / (s2 * P);                 /* RSS = ESS / (J N) */
}

double or_power_search(const double *loglik, int P, double phi, double d1,
                       int iters, double *rss_out)
{
    double llmax = -INFINITY;
    for (int n = 0; n < P; ++n) if (loglik[n] > llmax) llmax = loglik[n];
    double hi = 1.0 - phi;
    double r = rss_power(loglik, P, llmax, hi);
    if (r >= d1) { if (rss_out) *rss_out = r; return hi; }
    double lo = 0.0;
    for (int it = 0; it < iters; ++it) {
        double mid = 0.5 * (lo + hi);
        if (rss_power(loglik, P, llmax, mid) >= d1) lo = mid; else hi = mid;
    }
    if (rss_out) *rss_out = rss_power(loglik, P, llmax, hi);
    return hi;
}

/* ------------------------------- full run --------------------------------- */
static void gather_rows(double *a, const int32_t *src, int J, int N, int width, double *tmp)
{
    for (int j = 0; j < J; ++j)
        for (int n = 0; n < N; ++n) {
            size_t to = (size_t)j * N + n, from = (size_t)j * N + src[to];
            memcpy(tmp + to * width, a + from * width, sizeof(double) * (size_t)width);
        }
    memcpy(a, tmp, sizeof(double) * (size_t)J * N * width);
}

static int is_forced(const or_run_cfg *c, int s)
{
    if (c->burnin > 0 && s == c->burnin) return 1;    /* log score boundary */
    for (int i = 0; i < c->n_force; ++i) if (c->force_dates[i] == s) return 1;
    return 0;
}

/* Mean RNE of the test functions (EGARCH: g1..g3; otherwise the parameters). */
static double mean_rne(const or_model *m, const double *theta, const double *state,
                       int J, int N, double *gbuf)
{
    const int P = J * N;
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 0;
    const int nf = m->model == OR_EGARCH ? 3 : m->d;
    for (int n = 0; n < P; ++n) {
        if (m->model == OR_EGARCH) {
            double g[3];
            or_egarch_testfn(m, theta + (size_t)n * m->d, state + (size_t)n * ns, g);
            for (int f = 0; f < 3; ++f) gbuf[(size_t)f * P + n] = g[f];
        } else {
            for (int f = 0; f < nf; ++f) gbuf[(size_t)f * P + n] = theta[(size_t)n * m->d + f];
        }
    }
    double acc = 0.0;
    for (int f = 0; f < nf; ++f) {
        double mean, sd, nse, rne;
        or_moment(gbuf + (size_t)f * P, J, N, &mean, &sd, &nse, &rne);
        acc += rne;
    }
    return acc / nf;
}

int or_smc_run(const or_model *m, const double *y, const double *X, int T,
               const or_run_cfg *cfg, const double *theta0,
               double *theta, double *loglik, double *logprior, double *state,
               double *a_out, int *t_rec, double *phi_rec, int *r_rec,
               double *rss_rec, or_run_out *out)
{
    const int J = cfg->J, N = cfg->N, P = J * N, d = m->d;
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 1;
    const int power = cfg->tempering == 1;
    if (power && (cfg->burnin > 0 || cfg->pit_out)) {
        /* the log score and PIT walk the observations: data tempering only */
        memset(out, 0, sizeof *out);
        out->status = -5;
        return -5;
    }
    if (cfg->mutation == 2 && (cfg->replay || cfg->rec_L)) {
        /* a recorded design holds the factors L only, not the proposal means */
        memset(out, 0, sizeof *out);
        out->status = -4;
        return -4;
    }
    double *logw = calloc((size_t)P, sizeof(double));
    double *w = calloc((size_t)P, sizeof(double));
    double *tmp = calloc((size_t)P * (d > ns ? d : ns) + (size_t)P, sizeof(double));
    double *grad = calloc((size_t)P * d, sizeof(double));
    double *gbuf = calloc((size_t)P * (d > 3 ? d : 3), sizeof(double));
    double *lwj = calloc((size_t)J, sizeof(double));
    double *a_score = calloc((size_t)J, sizeof(double));
    int32_t *idx = calloc((size_t)P, sizeof(int32_t));
    double V[64 * 64], Sig[64 * 64], L[64 * 64], mean[64];
    memset(out, 0, sizeof(*out));

    /* Algorithm 1 step 1: particles from the prior (given), their prior density
     * and likelihood at the starting point of the tempering path. */
    memcpy(theta, theta0, sizeof(double) * (size_t)P * d);
    or_logprior_batch(m, theta, P, logprior);
    memset(state, 0, sizeof(double) * (size_t)P * ns);
    if (power) or_loglik_batch(m, y, X, T, theta, P, loglik, state, cfg->nthreads);
    else for (int n = 0; n < P; ++n) loglik[n] = 0.0;
    if (cfg->mutation == 1 && power)
        for (int n = 0; n < P; ++n)
            or_loglik_grad(m, y, X, T, theta + (size_t)n * d, grad + (size_t)n * d);
    for (int j = 0; j < J; ++j) a_out[j] = 0.0;

    double phi = 0.0, ltilde = 0.0;
    int t_prev = 0, h = cfg->h0_tenths, l = 0, status = 0;
    long replay_iter = 0;
    while ((power ? phi < 1.0 : t_prev < T) && l < cfg->max_cycles) {
        ++l;
        double rss = 1.0;
        int t_l = T, forced = 0;
        /* ---- C phase ---- */
        if (power) {
            double dphi;
            if (cfg->replay) {
                if (l > cfg->n_design) { status = -3; break; }
                dphi = cfg->design_x[l - 1] >= 1.0 ? 1.0 - phi : cfg->design_x[l - 1] - phi;
                double llmax = -INFINITY;
                for (int n = 0; n < P; ++n) if (loglik[n] > llmax) llmax = loglik[n];
                double s1 = 0.0, s2 = 0.0;
                for (int n = 0; n < P; ++n) {
                    if (loglik[n] == -INFINITY) continue;
                    double wv = exp(dphi * (loglik[n] - llmax));
                    s1 += wv;
                    s2 += wv * wv;
                }
                rss = s1 * s1 / (s2 * P);
            } else {
                dphi = or_power_search(loglik, P, phi, cfg->d1, cfg->bisect_iters, &rss);
            }
            int last = dphi >= 1.0 - phi;
            for (int n = 0; n < P; ++n)
                logw[n] = loglik[n] == -INFINITY ? -INFINITY : dphi * loglik[n];
            phi = last ? 1.0 : phi + dphi;
            forced = last;
            if (phi_rec) phi_rec[l - 1] = phi;
        } else {
            for (int n = 0; n < P; ++n) logw[n] = 0.0;          /* w(t_{l-1}) = 1 */
            int s = t_prev;
            for (;;) {
                ++s;
                double lwmax = -INFINITY, pit_num = 0.0, pit_den = 0.0;
                if (cfg->pit_out)
                    for (int n = 0; n < P; ++n) if (logw[n] > lwmax) lwmax = logw[n];
                for (int n = 0; n < P; ++n) {                   /* (C_phase_compute) */
                    /* w(s-1), the weight before y_s (Section 4.1 PIT) */
                    double wprev = cfg->pit_out && logw[n] != -INFINITY ? exp(logw[n] - lwmax) : 0.0;
                    double inc = or_loglik_range(m, y, X, s - 1, s, theta + (size_t)n * d,
                                                 state + (size_t)n * ns);
                    logw[n] += inc;
                    loglik[n] += inc;
                    if (cfg->pit_out) {
                        double es = or_obs_shock(m, y, X, s, theta + (size_t)n * d, state + (size_t)n * ns);
                        double ed = or_pit_shock(m, theta + (size_t)n * d, cfg->seed, (uint64_t)n, s);
                        pit_den += wprev;
                        if (ed <= es) pit_num += wprev;
                    }
                }
                if (cfg->pit_out) cfg->pit_out[s - 1] = pit_num / pit_den;
                rss = or_ess_log(logw, P) / P;
                if (cfg->replay) {
                    if (s >= (int)cfg->design_x[l - 1]) { forced = s == T; break; }
                    continue;
                }
                if (rss < cfg->d1) break;
                if (s == T || is_forced(cfg, s)) { forced = 1; break; }
            }
            t_l = s;
            if (t_l == T) forced = 1;
            if (t_rec) t_rec[l - 1] = t_l;
        }
        if (rss_rec) rss_rec[l - 1] = rss;
        /* Section 4.2: log wbar_j(l-1) and its products. */
        for (int j = 0; j < J; ++j) {
            lwj[j] = logsumexp(logw + (size_t)j * N, N) - log((double)N);
            a_out[j] += lwj[j];
            if (cfg->burnin > 0 && t_prev >= cfg->burnin) a_score[j] += lwj[j];  /* cycles after b */
        }
        ltilde += logsumexp(lwj, J) - log((double)J);
        /* ---- S phase ---- */
        for (int j = 0; j < J; ++j) {
            double mx = -INFINITY;
            for (int n = 0; n < N; ++n) if (logw[(size_t)j * N + n] > mx) mx = logw[(size_t)j * N + n];
            for (int n = 0; n < N; ++n)
                w[(size_t)j * N + n] = mx == -INFINITY ? 0.0 : exp(logw[(size_t)j * N + n] - mx);
        }
        const int scheme = cfg->resid == 1 ? 0 : cfg->resid == 0 ? 1 : cfg->resid;
        if (or_resample_scheme(w, J, N, scheme, cfg->seed, (uint64_t)l, idx) != 0) {
            status = -2;                                        /* degenerate group */
            break;
        }
        gather_rows(theta, idx, J, N, d, tmp);
        gather_rows(loglik, idx, J, N, 1, tmp);
        gather_rows(logprior, idx, J, N, 1, tmp);
        gather_rows(state, idx, J, N, ns, tmp);
        if (cfg->mutation == 1) gather_rows(grad, idx, J, N, d, tmp);
        /* ---- M phase ---- */
        const int Tm = power ? T : t_l;
        const double phim = power ? phi : 1.0;
        if (cfg->mutation == 1 && !power)
            for (int n = 0; n < P; ++n)
                or_loglik_grad(m, y, X, Tm, theta + (size_t)n * d, grad + (size_t)n * d);
        if (cfg->h_reset_each_cycle) h = cfg->h0_tenths;
        int R;
        if (cfg->replay) R = cfg->design_R[l - 1];
        else if (cfg->stop_rule == 0) R = rss < cfg->d2 ? cfg->kappa * cfg->rbar : cfg->rbar;
        else R = cfg->rmax;
        const double E = forced ? cfg->e2 : cfg->e1;
        int r;
        for (r = 0; r < R; ++r) {
            if (cfg->replay) {
                memcpy(L, cfg->design_L + (size_t)replay_iter * d * d, sizeof(double) * (size_t)d * d);
                ++replay_iter;
            } else {
                or_mean_cov(theta, P, d, mean, V);
                /* Sigma = h^2 V (random walk, MALA); V itself for the
                 * independent sampler, which has no step size */
                double hh = cfg->mutation == 2 ? 1.0 : (h / 10.0) * (h / 10.0);
                for (int i = 0; i < d * d; ++i) Sig[i] = hh * V[i];
                or_cholesky(Sig, d, L);
            }
            if (cfg->rec_L && out->metropolis_steps < cfg->rec_L_cap)
                memcpy(cfg->rec_L + (size_t)out->metropolis_steps * d * d, L, sizeof(double) * (size_t)d * d);
            long acc = cfg->mutation == 1
                ? or_mutate_mala(m, y, X, Tm, theta, loglik, logprior, grad, state, P, L,
                                 phim, cfg->seed, (uint64_t)l, (uint64_t)r, NULL, cfg->nthreads)
                : cfg->mutation == 2
                ? or_mutate_indep(m, y, X, Tm, theta, loglik, logprior, state, P, mean, L, phim,
                                  cfg->seed, (uint64_t)l, (uint64_t)r, NULL, cfg->nthreads)
                : or_mutate_rw(m, y, X, Tm, theta, loglik, logprior, state, P, L, phim,
                               cfg->seed, (uint64_t)l, (uint64_t)r, NULL, cfg->nthreads);
            out->metropolis_steps += 1;
            out->particle_obs_evals += (double)P * Tm;
            double rate = (double)acc / P;
            h = rate > cfg->acc_target ? h + 1 : h - 1;
            if (h < cfg->hmin_tenths) h = cfg->hmin_tenths;
            if (h > cfg->hmax_tenths) h = cfg->hmax_tenths;
            if (!cfg->replay && cfg->stop_rule == 1 && mean_rne(m, theta, state, J, N, gbuf) >= E) { ++r; break; }
        }
        if (r_rec) r_rec[l - 1] = r;
        t_prev = t_l;
    }
    out->cycles = l;
    or_log_ml(a_out, J, &out->log_ml, &out->log_ml_nse);
    out->log_score = out->log_score_nse = NAN;
    if (cfg->burnin > 0 && cfg->burnin < T) or_log_ml(a_score, J, &out->log_score, &out->log_score_nse);
    out->log_ml_tilde = ltilde;
    out->h_final_tenths = h;
    out->status = status;
    free(logw); free(w); free(tmp); free(grad); free(gbuf); free(lwj); free(idx); free(a_score);
    return status;
}
