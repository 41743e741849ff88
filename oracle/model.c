/*
 * Oracle model code: the EGARCH(K,I) model of Section 5.1 and a conjugate normal
 * linear regression used as a closed-form check.  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).  Plain double precision, written in the paper's order and notation.
 *
 * Passages followed:
 *   - parameters, priors and transforms: Table 1 and (EGARCH_tran1)-(EGARCH_tran2)
 *   - model: (EGARCH_mod1)-(EGARCH_mod2), mixture (normal_mixture)
 *   - per-observation density: the four evaluation steps of Section 5.1
 *   - test functions g1, g2, g3: Section 5.2
 * Readings where the paper is silent:
 *   - v_k1: the paper fixes v_k0 = 0 but not eps_0.  Default reading: there is no
 *     shock before the first observation, so v_k1 = alpha_k v_k0 = 0.  eps0_zero
 *     selects the alternative eps_0 = 0, i.e. v_k1 = -beta_k sqrt(2/pi).
 *   - I = 1: the normalisation forces p = 1, mu = 0, sigma = 1, so the mixture
 *     triple carries no information and is not a parameter (d = 2 + 3K).
 *   - gamma = 0 variants drop theta_5k (d = 2 + 2K for I = 1).
 *   - the log prior is the density kernel of Condition 1: the normalising
 *     constant of the theta_8i truncation is omitted (it cancels everywhere).
 *   - a non-finite log density is -inf (weight zero, proposal rejected).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_SQRT_2_OVER_PI 0.79788456080286535588  /* (2/pi)^{1/2} in (EGARCH_mod1) */
#define OR_LOG_2PI 1.83787706640934548356

int or_egarch_dim(int K, int I, int gamma)
{
    return 2 + 2 * K + (gamma ? K : 0) + (I >= 2 ? 3 * I : 0);
}

/* Table 1: mean, s.d. and transformation for theta_1 .. theta_8i.  Layout of the
 * full vector: theta_1, theta_2, theta_3k (k=1..K), theta_4k, [theta_5k],
 * [theta_6i (i=1..I), theta_7i, theta_8i]. */
void or_egarch_prior_table1(int K, int I, int gamma, double *mean, double *sd, double *lo)
{
    int j = 0;
    mean[j] = 0.0;        sd[j] = 1.0; lo[j] = -INFINITY; ++j;   /* theta_1  */
    mean[j] = log(0.01);  sd[j] = 1.0; lo[j] = -INFINITY; ++j;   /* theta_2  */
    for (int k = 0; k < K; ++k) { mean[j] = atanh(0.95); sd[j] = 1.0; lo[j] = -INFINITY; ++j; }
    for (int k = 0; k < K; ++k) { mean[j] = log(0.10);   sd[j] = 1.0; lo[j] = -INFINITY; ++j; }
    if (gamma)
        for (int k = 0; k < K; ++k) { mean[j] = 0.0; sd[j] = 0.2; lo[j] = -INFINITY; ++j; }
    if (I >= 2) {
        for (int i = 0; i < I; ++i) { mean[j] = 0.0; sd[j] = 1.0; lo[j] = -INFINITY; ++j; }
        for (int i = 0; i < I; ++i) { mean[j] = 0.0; sd[j] = 1.0; lo[j] = -INFINITY; ++j; }
        for (int i = 0; i < I; ++i) { mean[j] = 0.0; sd[j] = 1.0; lo[j] = -3.0;      ++j; }
    }
}

/* Fourth column of Table 1, then (EGARCH_tran1)-(EGARCH_tran2). */
void or_egarch_transform(int K, int I, int gamma, const double *th, or_egarch_par *q)
{
    int j = 0;
    q->mu_y = th[j++] / 1000.0;
    q->sigma_y = exp(th[j++]);
    for (int k = 0; k < K; ++k) q->alpha[k] = tanh(th[j++]);
    for (int k = 0; k < K; ++k) q->beta[k] = exp(th[j++]);
    for (int k = 0; k < K; ++k) q->gamma[k] = gamma ? th[j++] : 0.0;
    if (I == 1) {
        q->p[0] = 1.0; q->mu[0] = 0.0; q->sig[0] = 1.0;
        return;
    }
    double pstar[8], mustar[8], sigstar[8];
    for (int i = 0; i < I; ++i) pstar[i] = tanh(th[j++]) + 1.0;
    for (int i = 0; i < I; ++i) mustar[i] = th[j++];
    for (int i = 0; i < I; ++i) sigstar[i] = exp(th[j++]);
    double psum = 0.0;
    for (int i = 0; i < I; ++i) psum += pstar[i];
    for (int i = 0; i < I; ++i) q->p[i] = pstar[i] / psum;
    double pmu = 0.0;
    for (int i = 0; i < I; ++i) pmu += q->p[i] * mustar[i];
    double mu2[8], s = 0.0;
    for (int i = 0; i < I; ++i) {
        mu2[i] = mustar[i] - pmu;
        s += q->p[i] * (mu2[i] * mu2[i] + sigstar[i] * sigstar[i]);
    }
    double c = 1.0 / sqrt(s);
    for (int i = 0; i < I; ++i) {
        q->mu[i] = c * mu2[i];
        q->sig[i] = c * sigstar[i];
    }
}

void or_full_theta(const or_model *m, const double *theta, double *full)
{
    if (!m->free_idx) {
        memcpy(full, theta, sizeof(double) * (size_t)m->d_full);
        return;
    }
    for (int i = 0; i < m->d_full; ++i) full[i] = m->theta_fixed ? m->theta_fixed[i] : 0.0;
    for (int k = 0; k < m->d; ++k) full[m->free_idx[k]] = theta[k];
}

double or_logprior(const or_model *m, const double *theta)
{
    double lp = 0.0;
    for (int k = 0; k < m->d; ++k) {
        if (theta[k] < m->prior_lo[k] || !isfinite(theta[k])) return -INFINITY;
        double z = (theta[k] - m->prior_mean[k]) / m->prior_sd[k];
        lp += -0.5 * OR_LOG_2PI - log(m->prior_sd[k]) - 0.5 * z * z;
    }
    return lp;
}

void or_logprior_grad(const or_model *m, const double *theta, double *grad)
{
    for (int k = 0; k < m->d; ++k) {
        double s = m->prior_sd[k];
        grad[k] = -(theta[k] - m->prior_mean[k]) / (s * s);
    }
}

/* log of the mixture density (normal_mixture) at eps, as a max-shifted sum. */
static double log_mixture(const or_egarch_par *q, int I, double eps)
{
    double x[8], xmax = -INFINITY;
    for (int i = 0; i < I; ++i) {
        double z = (eps - q->mu[i]) / q->sig[i];
        x[i] = log(q->p[i]) - log(q->sig[i]) - 0.5 * z * z;
        if (x[i] > xmax) xmax = x[i];
    }
    double s = 0.0;
    for (int i = 0; i < I; ++i) s += exp(x[i] - xmax);
    return -0.5 * OR_LOG_2PI + xmax + log(s);
}

/* Steps 2-4 of Section 5.1 for observations t0+1 .. t1 (1-based), continuing
 * from state = (v_1..v_K, eps_{t0}).  Returns sum of log p(y_t | y_{1:t-1}). */
static double egarch_range(const or_model *m, const or_egarch_par *q, const double *y,
                           int t0, int t1, double *state, double *lt)
{
    const int K = m->K, I = m->I;
    double v[8], eps = 0.0;
    if (t0 == 0) {
        for (int k = 0; k < K; ++k) v[k] = 0.0;      /* v_k0 = 0 */
    } else {
        for (int k = 0; k < K; ++k) v[k] = state[k];
        eps = state[K];
    }
    double sum = 0.0;
    for (int t = t0 + 1; t <= t1; ++t) {
        /* Step 2: (EGARCH_mod1). */
        for (int k = 0; k < K; ++k) {
            if (t == 1) {
                v[k] = m->eps0_zero ? q->beta[k] * (0.0 - OR_SQRT_2_OVER_PI) : 0.0;
            } else {
                v[k] = q->alpha[k] * v[k] + q->beta[k] * (fabs(eps) - OR_SQRT_2_OVER_PI)
                     + q->gamma[k] * eps;
            }
        }
        /* Step 3: h_t and eps_t. */
        double vs = 0.0;
        for (int k = 0; k < K; ++k) vs += v[k];
        double h = q->sigma_y * exp(vs / 2.0);
        eps = (y[t - 1] - q->mu_y) / h;
        /* Step 4: (2 pi)^{-1/2} h^{-1} sum_i p_i sigma_i^{-1} exp(-(eps-mu_i)^2 / 2 sigma_i^2). */
        double l = log_mixture(q, I, eps) - log(h);
        if (!isfinite(l)) l = -INFINITY;
        if (lt) lt[t - 1 - t0] = l;
        sum += l;
    }
    if (state) {
        for (int k = 0; k < K; ++k) state[k] = v[k];
        state[K] = eps;
    }
    return sum;
}

static double linreg_range(const or_model *m, const double *full, const double *y,
                           const double *X, int t0, int t1, double *lt)
{
    const int p = m->p;
    const double s2 = m->sigma * m->sigma;
    double sum = 0.0;
    for (int t = t0 + 1; t <= t1; ++t) {
        double mean = 0.0;
        for (int i = 0; i < p; ++i) mean += X[(size_t)(t - 1) * p + i] * full[i];
        double r = y[t - 1] - mean;
        double l = -0.5 * OR_LOG_2PI - 0.5 * log(s2) - 0.5 * r * r / s2;
        if (lt) lt[t - 1 - t0] = l;
        sum += l;
    }
    return sum;
}

double or_loglik_range(const or_model *m, const double *y, const double *X,
                       int t0, int t1, const double *theta, double *state)
{
    double full[64];
    or_full_theta(m, theta, full);
    double s;
    if (m->model == OR_LINREG) {
        s = linreg_range(m, full, y, X, t0, t1, NULL);
    } else {
        or_egarch_par q;
        or_egarch_transform(m->K, m->I, m->gamma, full, &q);
        s = egarch_range(m, &q, y, t0, t1, state, NULL);
    }
    return isnan(s) ? -INFINITY : s;
}

double or_loglik(const or_model *m, const double *y, const double *X, int T,
                 const double *theta, double *state_out)
{
    double st[9] = {0};
    double s = or_loglik_range(m, y, X, 0, T, theta, st);
    if (state_out && m->model == OR_EGARCH)
        for (int k = 0; k <= m->K; ++k) state_out[k] = st[k];
    return s;
}

void or_loglik_terms(const or_model *m, const double *y, const double *X, int T,
                     const double *theta, double *lt)
{
    double full[64];
    or_full_theta(m, theta, full);
    if (m->model == OR_LINREG) {
        linreg_range(m, full, y, X, 0, T, lt);
    } else {
        or_egarch_par q;
        or_egarch_transform(m->K, m->I, m->gamma, full, &q);
        double st[9];
        egarch_range(m, &q, y, 0, T, st, lt);
    }
}

/* Section 5.2 test functions at the end state (v_kt, eps_t), t >= 1:
 *   g1 = log sigma_Y + sum_k v_kt / 2
 *   g2 = E(eps^3 | theta) = sum_i p_i (mu_i^3 + 3 mu_i sigma_i^2)
 *   g3 = P(Y_{t+1} < -0.03 | theta, y_{1:t}) = sum_i p_i Phi(((-0.03 - mu_Y)/h_{t+1} - mu_i)/sigma_i) */
void or_egarch_testfn(const or_model *m, const double *theta, const double *state, double g[3])
{
    double full[64];
    or_full_theta(m, theta, full);
    or_egarch_par q;
    or_egarch_transform(m->K, m->I, m->gamma, full, &q);
    const int K = m->K, I = m->I;
    double vs = 0.0, vnext = 0.0;
    double eps = state[K];
    for (int k = 0; k < K; ++k) {
        vs += state[k];
        vnext += q.alpha[k] * state[k] + q.beta[k] * (fabs(eps) - OR_SQRT_2_OVER_PI)
               + q.gamma[k] * eps;
    }
    g[0] = log(q.sigma_y) + vs / 2.0;
    double s3 = 0.0;
    for (int i = 0; i < I; ++i) s3 += q.p[i] * (pow(q.mu[i], 3) + 3.0 * q.mu[i] * q.sig[i] * q.sig[i]);
    g[1] = s3;
    double hn = q.sigma_y * exp(vnext / 2.0);
    double x = (-0.03 - q.mu_y) / hn;
    double pr = 0.0;
    for (int i = 0; i < I; ++i) pr += q.p[i] * 0.5 * erfc(-((x - q.mu[i]) / q.sig[i]) / sqrt(2.0));
    g[2] = pr;
}

/* ---------------- forward-mode (dual number) gradient ---------------------- */
typedef struct { double v, d; } dual;
static dual D(double v, double d) { dual r = {v, d}; return r; }
static dual dadd(dual a, dual b) { return D(a.v + b.v, a.d + b.d); }
static dual dsub(dual a, dual b) { return D(a.v - b.v, a.d - b.d); }
static dual dmul(dual a, dual b) { return D(a.v * b.v, a.d * b.v + a.v * b.d); }
static dual ddiv(dual a, dual b) { return D(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static dual dscale(dual a, double s) { return D(a.v * s, a.d * s); }
static dual dexp(dual a) { double e = exp(a.v); return D(e, e * a.d); }
static dual dlog(dual a) { return D(log(a.v), a.d / a.v); }
static dual dtanh(dual a) { double t = tanh(a.v); return D(t, (1.0 - t * t) * a.d); }
static dual dsqrt(dual a) { double s = sqrt(a.v); return D(s, a.d / (2.0 * s)); }
static dual dabs(dual a) { return a.v < 0 ? D(-a.v, -a.d) : a; }

typedef struct {
    dual mu_y, sigma_y, alpha[8], beta[8], gamma[8], p[8], mu[8], sig[8];
} dpar;

static void dtransform(int K, int I, int gam, const dual *th, dpar *q)
{
    int j = 0;
    q->mu_y = dscale(th[j++], 1.0 / 1000.0);
    q->sigma_y = dexp(th[j++]);
    for (int k = 0; k < K; ++k) q->alpha[k] = dtanh(th[j++]);
    for (int k = 0; k < K; ++k) q->beta[k] = dexp(th[j++]);
    for (int k = 0; k < K; ++k) q->gamma[k] = gam ? th[j++] : D(0.0, 0.0);
    if (I == 1) {
        q->p[0] = D(1, 0); q->mu[0] = D(0, 0); q->sig[0] = D(1, 0);
        return;
    }
    dual pstar[8], mustar[8], sigstar[8];
    for (int i = 0; i < I; ++i) pstar[i] = dadd(dtanh(th[j++]), D(1.0, 0.0));
    for (int i = 0; i < I; ++i) mustar[i] = th[j++];
    for (int i = 0; i < I; ++i) sigstar[i] = dexp(th[j++]);
    dual psum = D(0, 0);
    for (int i = 0; i < I; ++i) psum = dadd(psum, pstar[i]);
    for (int i = 0; i < I; ++i) q->p[i] = ddiv(pstar[i], psum);
    dual pmu = D(0, 0);
    for (int i = 0; i < I; ++i) pmu = dadd(pmu, dmul(q->p[i], mustar[i]));
    dual mu2[8], s = D(0, 0);
    for (int i = 0; i < I; ++i) {
        mu2[i] = dsub(mustar[i], pmu);
        s = dadd(s, dmul(q->p[i], dadd(dmul(mu2[i], mu2[i]), dmul(sigstar[i], sigstar[i]))));
    }
    dual c = ddiv(D(1, 0), dsqrt(s));
    for (int i = 0; i < I; ++i) {
        q->mu[i] = dmul(c, mu2[i]);
        q->sig[i] = dmul(c, sigstar[i]);
    }
}

static double dual_loglik(const or_model *m, const double *y, const double *X, int T,
                          const dual *full, double *val)
{
    dual sum = D(0, 0);
    if (m->model == OR_LINREG) {
        double s2 = m->sigma * m->sigma;
        for (int t = 0; t < T; ++t) {
            dual mean = D(0, 0);
            for (int i = 0; i < m->p; ++i) mean = dadd(mean, dscale(full[i], X[(size_t)t * m->p + i]));
            dual r = dsub(D(y[t], 0), mean);
            dual l = dsub(D(-0.5 * OR_LOG_2PI - 0.5 * log(s2), 0), dscale(dmul(r, r), 0.5 / s2));
            sum = dadd(sum, l);
        }
        *val = sum.v;
        return sum.d;
    }
    const int K = m->K, I = m->I;
    dpar q;
    dtransform(K, I, m->gamma, full, &q);
    dual v[8], eps = D(0, 0);
    for (int k = 0; k < K; ++k) v[k] = D(0, 0);
    for (int t = 1; t <= T; ++t) {
        for (int k = 0; k < K; ++k) {
            if (t == 1) {
                v[k] = m->eps0_zero ? dscale(q.beta[k], -OR_SQRT_2_OVER_PI) : D(0, 0);
            } else {
                v[k] = dadd(dadd(dmul(q.alpha[k], v[k]),
                                 dmul(q.beta[k], dsub(dabs(eps), D(OR_SQRT_2_OVER_PI, 0)))),
                            dmul(q.gamma[k], eps));
            }
        }
        dual vs = D(0, 0);
        for (int k = 0; k < K; ++k) vs = dadd(vs, v[k]);
        dual h = dmul(q.sigma_y, dexp(dscale(vs, 0.5)));
        eps = ddiv(dsub(D(y[t - 1], 0), q.mu_y), h);
        dual x[8];
        double xmax = -INFINITY;
        for (int i = 0; i < I; ++i) {
            dual z = ddiv(dsub(eps, q.mu[i]), q.sig[i]);
            x[i] = dsub(dsub(dlog(q.p[i]), dlog(q.sig[i])), dscale(dmul(z, z), 0.5));
            if (x[i].v > xmax) xmax = x[i].v;
        }
        dual s = D(0, 0);
        for (int i = 0; i < I; ++i) s = dadd(s, dexp(dsub(x[i], D(xmax, 0))));
        dual l = dsub(dadd(D(-0.5 * OR_LOG_2PI + xmax, 0), dlog(s)), dlog(h));
        sum = dadd(sum, l);
    }
    *val = sum.v;
    return sum.d;
}

double or_loglik_grad(const or_model *m, const double *y, const double *X, int T,
                      const double *theta, double *grad)
{
    double full[64];
    or_full_theta(m, theta, full);
    double val = 0.0;
    for (int j = 0; j < m->d; ++j) {
        dual fd[64];
        for (int i = 0; i < m->d_full; ++i) fd[i] = D(full[i], 0.0);
        int pos = m->free_idx ? m->free_idx[j] : j;
        fd[pos].d = 1.0;
        grad[j] = dual_loglik(m, y, X, T, fd, &val);
    }
    if (m->d == 0) {
        dual fd[64];
        for (int i = 0; i < m->d_full; ++i) fd[i] = D(full[i], 0.0);
        dual_loglik(m, y, X, T, fd, &val);
    }
    return isnan(val) ? -INFINITY : val;
}

void or_loglik_batch(const or_model *m, const double *y, const double *X, int T,
                     const double *theta, int P, double *loglik, double *state,
                     int nthreads)
{
    const int ns = m->model == OR_EGARCH ? m->K + 1 : 0;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int n = 0; n < P; ++n) {
        double st[9] = {0};
        loglik[n] = or_loglik(m, y, X, T, theta + (size_t)n * m->d, st);
        if (state && ns)
            for (int k = 0; k < ns; ++k) state[(size_t)n * ns + k] = st[k];
    }
}

void or_logprior_batch(const or_model *m, const double *theta, int P, double *lp)
{
    for (int n = 0; n < P; ++n) lp[n] = or_logprior(m, theta + (size_t)n * m->d);
}
