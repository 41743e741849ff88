"""Pins for the oracle's estimators and C/S/M phases, and for full runs.

Closed forms: conjugate normal regression (exact log marginal likelihood and
posterior moments); a one-parameter EGARCH model by dense quadrature.
Distributional facts: Proposition 1 (chi-square / t limits of the group-based
variance estimate), the resampler's expected counts, invariance of the
Metropolis kernels.  Library routines: numpy.cov, numpy.linalg.cholesky."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1304_4334_gb300 import inputs as I
from tests.golden_io import defaults


def test_defaults_fixture_matches_runner_defaults():
    d = defaults()
    r = O.DEFAULT_RUN
    assert (r["d1"], r["d2"], r["rbar"], r["kappa"]) == (d["D1"], d["D2"], d["Rbar"], d["kappa"])
    assert (r["e1"], r["e2"], r["rmax"]) == (d["E1"], d["E2"], d["Rmax"])
    assert r["h0_tenths"] / 10 == d["h0"] and r["hmin_tenths"] / 10 == d["h_min"]
    assert r["hmax_tenths"] / 10 == d["h_max"] and r["acc_target"] == d["acc_target"]


# ----------------------------------------------------------------- estimators
def test_moment_prop1_chi_square_and_t():
    """For iid draws Condition 5 holds exactly with v = var g; Proposition 1 says
    (J-1) vhat / v ~ chi2(J-1) and the standardized error ~ t(J-1)."""
    rng = np.random.default_rng(0)
    J, N = 8, 64
    chi, tt, rne = [], [], []
    for _ in range(800):
        g = rng.standard_normal(J * N)
        mean, sd, nse, r = O.moment(g, J, N)
        vhat = nse ** 2 * J * N
        chi.append((J - 1) * vhat / 1.0)
        tt.append(mean / nse)
        rne.append(r)
    assert stats.kstest(chi, stats.chi2(J - 1).cdf).pvalue > 1e-3
    assert stats.kstest(tt, stats.t(J - 1).cdf).pvalue > 1e-3
    assert 0.8 < np.median(rne) < 1.25


def test_moment_special_cases():
    J, N = 4, 5
    g = np.repeat(np.arange(J, dtype=float), N)        # within-group constant
    mean, sd, nse, rne = O.moment(g, J, N)
    assert mean == pytest.approx(1.5)
    assert nse == pytest.approx(math.sqrt(np.var(np.arange(J), ddof=1) / J))
    g2 = np.tile(np.arange(N, dtype=float), J)         # identical group means
    assert O.moment(g2, J, N)[2] == 0.0 and O.moment(g2, J, N)[3] == np.inf


def test_ess_special_cases():
    assert O.ess_log(np.zeros(100)) == pytest.approx(100, rel=1e-14)
    lw = np.full(50, -np.inf)
    lw[7] = 3.0
    assert O.ess_log(lw) == pytest.approx(1.0)
    lw = np.full(40, -np.inf)
    lw[:13] = -2.5
    assert O.ess_log(lw) == pytest.approx(13, rel=1e-14)


def test_log_ml_special_cases():
    a = np.full(6, -123.4)
    lm, nse = O.log_ml(a)
    assert lm == pytest.approx(-123.4, rel=1e-15) and nse == 0.0
    a = np.log(np.array([1.0, 2.0, 3.0, 6.0]))
    lm, nse = O.log_ml(a)
    assert lm == pytest.approx(math.log(3.0), rel=1e-14)
    assert nse == pytest.approx(math.sqrt(np.var([1, 2, 3, 6], ddof=1) / 4) / 3.0, rel=1e-13)


# -------------------------------------------------------------------- S phase
def _counts(idx, N):
    return np.stack([np.bincount(row, minlength=N) for row in idx])


def test_resample_counts_and_residual_floor():
    rng = np.random.default_rng(1)
    J, N = 5, 200
    w = rng.gamma(0.5, size=J * N)
    idx = O.resample(w, J, N, resid=True, seed=3, cycle=1)
    c = _counts(idx, N)
    assert np.all(c.sum(axis=1) == N)
    wt = w.reshape(J, N) / w.reshape(J, N).sum(axis=1, keepdims=True)
    assert np.all(c >= np.floor(N * wt - 1e-9))        # deterministic part of residual
    assert np.all(c <= np.floor(N * wt) + N)           # trivially bounded
    assert np.all(np.diff(idx, axis=1) >= 0)           # expansion is in particle order


def test_resample_degenerate_and_uniform():
    N = 64
    w = np.zeros(N)
    w[17] = 0.3
    assert np.all(O.resample(w, 1, N, resid=True, seed=1, cycle=0) == 17)
    assert np.all(O.resample(w, 1, N, resid=False, seed=1, cycle=0) == 17)
    assert np.array_equal(O.resample(np.ones(N), 1, N, resid=True)[0], np.arange(N))
    with pytest.raises(ValueError):
        O.resample(np.zeros(N), 1, N)


@pytest.mark.parametrize("resid", [True, False])
def test_resample_expected_counts(resid):
    rng = np.random.default_rng(2)
    N = 16
    w = rng.gamma(1.0, size=N)
    wt = w / w.sum()
    reps = 4000
    tot = np.zeros(N)
    for cyc in range(reps):
        tot += np.bincount(O.resample(w, 1, N, resid=resid, seed=11, cycle=cyc)[0], minlength=N)
    expected = reps * N * wt
    # chi-square on the mean counts; residual resampling has smaller variance,
    # so a multinomial-variance chi-square is conservative for it.
    chi2 = np.sum((tot - expected) ** 2 / expected)
    assert chi2 < stats.chi2(N - 1).ppf(0.999)


# ----------------------------------------------------- covariance, Cholesky
def test_mean_cov_and_cholesky_against_numpy():
    rng = np.random.default_rng(5)
    th = rng.normal(size=(500, 6)) @ rng.normal(size=(6, 6)) + 3.0
    m, c = O.mean_cov(th)
    np.testing.assert_allclose(m, th.mean(axis=0), rtol=1e-13)
    np.testing.assert_allclose(c, np.cov(th.T), rtol=1e-11)
    L, z = O.cholesky(c)
    assert z == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(c), rtol=1e-11, atol=1e-13)


def test_cholesky_rank_deficient_zeroes_column():
    A = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 9.0]])
    L, z = O.cholesky(A)
    assert z == 1
    np.testing.assert_allclose(L @ L.T, A, atol=1e-12)


# -------------------------------------------------------------------- C phase
def test_power_search_hits_target_rss():
    rng = np.random.default_rng(7)
    ll = rng.normal(-1000, 30, 4096)
    dphi, rss = O.power_search(ll, 0.0, 0.5)
    w = np.exp(dphi * (ll - ll.max()))
    assert (w.sum() ** 2 / (w ** 2).sum()) / len(ll) == pytest.approx(rss, rel=1e-12)
    assert rss < 0.5 and rss == pytest.approx(0.5, abs=1e-9)
    w2 = np.exp(0.999999 * dphi * (ll - ll.max()))
    assert (w2.sum() ** 2 / (w2 ** 2).sum()) / len(ll) >= 0.5 - 1e-6
    # flat likelihood: RSS stays 1, the whole remaining power is taken
    assert O.power_search(np.full(100, -5.0), 0.3, 0.5)[0] == pytest.approx(0.7)


# -------------------------------------------------------- conjugate regression
def _linreg_problem(T=60, seed=3):
    beta = np.array([0.5, -1.0, 2.0])
    sigma = 1.0
    X, y = I.linreg_data(T, beta, sigma, seed=seed)
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    V0 = np.diag(s0 ** 2)
    lml = stats.multivariate_normal(X @ m0, sigma ** 2 * np.eye(T) + X @ V0 @ X.T).logpdf(y)
    Vn = np.linalg.inv(np.linalg.inv(V0) + X.T @ X / sigma ** 2)
    mn = Vn @ (np.linalg.inv(V0) @ m0 + X.T @ y / sigma ** 2)
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=sigma, prior_mean=m0, prior_sd=s0)
    return spec, X, y, lml, mn, Vn, (m0, s0)


def test_rw_kernel_leaves_posterior_invariant():
    spec, X, y, _, mn, Vn, _ = _linreg_problem()
    rng = np.random.default_rng(11)
    P = 20000
    th = rng.multivariate_normal(mn, Vn, size=P)
    ll = O.loglik(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    L = np.linalg.cholesky(0.8 ** 2 * Vn)
    st = np.zeros((P, 1))
    for it in range(5):
        th, ll, lp, st, acc, nacc = O.mutate_rw(spec, y, th, ll, lp, st, L, 1.0, 5, 1, it, X=X)
    assert 0.2 < nacc / P < 0.8
    se = np.sqrt(np.diag(Vn) / P) * 3     # particles stay (correlated) posterior draws
    assert np.all(np.abs(th.mean(axis=0) - mn) < 4 * se)
    np.testing.assert_allclose(np.cov(th.T), Vn, rtol=0.1, atol=0.05 * np.abs(Vn).max())


def test_mala_kernel_leaves_posterior_invariant():
    spec, X, y, _, mn, Vn, _ = _linreg_problem()
    rng = np.random.default_rng(12)
    P = 8000
    th = rng.multivariate_normal(mn, Vn, size=P)
    ll, g = O.loglik_grad(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    L = np.linalg.cholesky(1.2 ** 2 * Vn)
    st = np.zeros((P, 1))
    for it in range(4):
        th, ll, lp, g, st, acc, nacc = O.mutate_mala(spec, y, th, ll, lp, g, st, L, 1.0, 6, 1, it, X=X)
    assert nacc / P > 0.3
    se = np.sqrt(np.diag(Vn) / P) * 3
    assert np.all(np.abs(th.mean(axis=0) - mn) < 4 * se)
    np.testing.assert_allclose(np.cov(th.T), Vn, rtol=0.1, atol=0.05 * np.abs(Vn).max())
    # the stored gradient follows the accepted particle
    _, g2 = O.loglik_grad(spec, y, th[:50], X=X)
    np.testing.assert_allclose(g[:50], g2, rtol=1e-12)


@pytest.mark.parametrize("tempering,mutation", [(1, 0), (0, 0), (1, 1)])
def test_full_run_linreg_matches_closed_form(tempering, mutation):
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 512
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=21)
    r = O.smc_run(spec, y, th0, J, N, X=X, tempering=tempering, mutation=mutation,
                  seed=5 + tempering + 2 * mutation,
                  acc_target=0.25 if mutation == 0 else 0.5)
    assert r["status"] == 0
    z = (r["log_ml"] - lml) / r["log_ml_nse"]
    assert abs(z) < 3.5, (r["log_ml"], lml, r["log_ml_nse"])
    assert abs(r["log_ml_tilde"] - lml) < 5 * r["log_ml_nse"] + 0.02
    for i in range(3):
        mean, sd, nse, rne = O.moment(r["theta"][:, i], J, N)
        assert abs(mean - mn[i]) < 3.5 * nse + 1e-4, (i, mean, mn[i], nse)
        assert sd == pytest.approx(math.sqrt(Vn[i, i]), rel=0.08)
    if tempering == 0:
        assert r["t"][-1] == len(y) and np.all(np.diff(r["t"]) > 0)
    else:
        assert r["phi"][-1] == 1.0 and np.all(np.diff(r["phi"]) > 0)


def test_rne_stopping_rule_runs_and_respects_cap():
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 256
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=22)
    r = O.smc_run(spec, y, th0, J, N, X=X, stop_rule=1, rmax=30, seed=9)
    assert r["status"] == 0 and np.all(r["R"] >= 1) and np.all(r["R"] <= 30)
    assert abs(r["log_ml"] - lml) < 4 * r["log_ml_nse"] + 0.02


def test_full_run_one_parameter_egarch_matches_quadrature():
    """Only theta_2 (log sigma_Y) is free; the rest is fixed at the truth.
    log p(y) = log int N(theta_2; log .01, 1) p(y|theta_2) dtheta_2 by dense
    quadrature with the oracle's likelihood."""
    tr = I.EgarchTruth(0.0, 0.01, (0.95,), (0.12,), (-0.05,))
    y = I.simulate_egarch(tr, 300, seed=31)
    th_true = I.theta_of_truth(tr)
    spec = O.ModelSpec(K=1, I=1, gamma=True, free_idx=[1], theta_fixed=th_true)
    grid = np.linspace(math.log(0.01) - 2.0, math.log(0.01) + 2.0, 40001)
    lj = O.loglik(spec, y, grid[:, None]) + O.logprior(spec, grid[:, None])
    mx = lj.max()
    wq = np.exp(lj - mx)
    dx = grid[1] - grid[0]
    Z = integrate_simpson(wq, dx)
    lml = mx + math.log(Z)
    pmean = integrate_simpson(wq * grid, dx) / Z
    assert wq[0] < 1e-20 and wq[-1] < 1e-20           # the grid covers the mass
    J, N = 8, 256
    th0 = I.draw_prior([math.log(0.01)], [1.0], [-np.inf], J * N, seed=41)
    for tempering in (1, 0):
        r = O.smc_run(spec, y, th0, J, N, tempering=tempering, seed=3 + tempering)
        assert abs(r["log_ml"] - lml) < 3.5 * r["log_ml_nse"] + 0.01, (tempering, r["log_ml"], lml)
        mean, sd, nse, rne = O.moment(r["theta"][:, 0], J, N)
        assert abs(mean - pmean) < 3.5 * nse + 1e-4


def integrate_simpson(f, dx):
    from scipy.integrate import simpson
    return simpson(f, dx=dx)


@pytest.mark.slow
def test_nse_coverage_over_seeds():
    """Proposition 1 (p1B) for the hybrid-free adaptive run: the standardized
    error of the posterior mean is about t(J-1); check two-sided 95% coverage
    over independent seeds with a binomial tolerance."""
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem(T=40, seed=8)
    J, N = 8, 256
    tq = stats.t(J - 1).ppf(0.975)
    hits_m, hits_ml, n = 0, 0, 120
    for s in range(n):
        th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=1000 + s)
        r = O.smc_run(spec, y, th0, J, N, X=X, seed=500 + s, rbar=10)
        mean, sd, nse, rne = O.moment(r["theta"][:, 0], J, N)
        hits_m += abs(mean - mn[0]) < tq * nse
        hits_ml += abs(r["log_ml"] - lml) < tq * r["log_ml_nse"]
    # 95% nominal; binomial(120, .95) has sd 2.4, so >= 102 is about 4 sd low
    assert hits_m >= 102, hits_m
    assert hits_ml >= 96, hits_ml


def test_resample_large_group_many_residual_draws():
    """N = 8192 with one dominant weight: almost every count is fractional, so
    nearly N residual draws are made and the residual total is near Q N."""
    N = 8192
    w = np.full(N, 1e-3)
    w[5] = 1.0
    idx = O.resample(w, 1, N, resid=True, seed=2, cycle=3)[0]
    c = np.bincount(idx, minlength=N)
    assert c.sum() == N
    wt = w / w.sum()
    assert c[5] >= np.floor(N * wt[5])
    # the residual draws spread over the small particles in proportion
    others = np.delete(c, 5)
    exp_other = N * wt[0] - np.floor(N * wt[0])
    assert abs(others.mean() - (N * wt[0])) < 0.1 + 4 * np.sqrt(exp_other / (N - 1))


# ---------------------------------------------------------- Algorithm 3 (hybrid)
@pytest.mark.parametrize("tempering", [1, 0])
def test_hybrid_replay_same_seed_reproduces_the_adaptive_run(tempering):
    """Replaying the recorded design with the same random numbers is the
    adaptive run itself: same cycle ends, iterations and proposal scales."""
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 256
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=31)
    a = O.smc_run(spec, y, th0, J, N, X=X, tempering=tempering, seed=9, record=True)
    dsg = a["design"]
    assert len(dsg["x"]) == a["cycles"] and dsg["L"].shape[0] == a["metropolis_steps"]
    b = O.smc_run(spec, y, th0, J, N, X=X, tempering=tempering, seed=9, design=dsg)
    assert b["cycles"] == a["cycles"] and np.array_equal(b["R"], a["R"])
    assert b["log_ml"] == pytest.approx(a["log_ml"], abs=1e-9)
    np.testing.assert_allclose(b["theta"], a["theta"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("tempering", [1, 0])
def test_hybrid_second_run_matches_closed_form(tempering):
    """Algorithm 3: keep the design of an adaptive run, rerun non-adaptively
    with a new seed; the second run's estimates satisfy Condition 5."""
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 512
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=32)
    a = O.smc_run(spec, y, th0, J, N, X=X, tempering=tempering, seed=10, record=True)
    th1 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=33)
    b = O.smc_run(spec, y, th1, J, N, X=X, tempering=tempering, seed=11, design=a["design"])
    assert b["status"] == 0 and b["cycles"] == a["cycles"]
    if tempering == 1:
        np.testing.assert_allclose(b["phi"], a["phi"], rtol=0, atol=1e-12)
    else:
        assert np.array_equal(b["t"], a["t"])
    # J = 8 groups: standardized errors are t(7) (Proposition 1); 4.0 is its
    # two-sided 99.5% point
    assert abs(b["log_ml"] - lml) < 4.0 * b["log_ml_nse"] + 0.02
    for i in range(3):
        mean, sd, nse, rne = O.moment(b["theta"][:, i], J, N)
        assert abs(mean - mn[i]) < 4.0 * nse + 1e-4


# ----------------------------------------- stratified / systematic resampling
@pytest.mark.parametrize("scheme", [O.STRATIFIED, O.SYSTEMATIC])
def test_stratified_systematic_properties(scheme):
    rng = np.random.default_rng(4)
    N = 64
    w = rng.gamma(0.7, size=N)
    wt = w / w.sum()
    reps = 3000
    tot = np.zeros(N)
    for cyc in range(reps):
        idx = O.resample_scheme(w, 1, N, scheme, seed=3, cycle=cyc)[0]
        assert np.all(np.diff(idx) >= 0)
        c = np.bincount(idx, minlength=N)
        # both schemes give floor(N w~) or ceil(N w~) copies of every particle
        # (stratified up to one more or less where strata straddle)
        lo = np.floor(N * wt) - (0 if scheme == O.SYSTEMATIC else 1)
        hi = np.ceil(N * wt) + (0 if scheme == O.SYSTEMATIC else 1)
        assert np.all(c >= lo - 1e-9) and np.all(c <= hi + 1e-9)
        tot += c
    # unbiased: E[count] = N w~
    se = np.sqrt(np.maximum(N * wt * (1 - wt), 1e-3) / reps)
    assert np.all(np.abs(tot / reps - N * wt) < 6 * se + 1e-3)


@pytest.mark.parametrize("scheme", [2, 3])
def test_full_run_with_stratified_and_systematic(scheme):
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 512
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=41)
    r = O.smc_run(spec, y, th0, J, N, X=X, resid=scheme, seed=13)
    assert r["status"] == 0
    assert abs(r["log_ml"] - lml) < 4.0 * r["log_ml_nse"] + 0.02


# ------------------------------------------- independent Gaussian sampler
def test_indep_with_exact_posterior_proposal_accepts_every_draw():
    """With q equal to the (Gaussian) posterior the Metropolis ratio is exactly
    1, so every proposal is accepted and lands at mbar + L z (Section 3.3's
    independent sampler; a sign slip in the q correction rejects many)."""
    spec, X, y, _, mn, Vn, _ = _linreg_problem()
    rng = np.random.default_rng(31)
    P = 3000
    th = rng.multivariate_normal(mn + 0.3, 2.0 * Vn, size=P)
    ll = O.loglik(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    L = np.linalg.cholesky(Vn)
    st = np.zeros((P, 1))
    th2, ll2, lp2, _, acc, n = O.mutate_indep(spec, y, th, ll, lp, st, mn, L, 1.0, 7, 2, 3, X=X)
    assert n == P and acc.all()
    for p in (0, 17, P - 1):
        z = O.philox_normals(7, p, 3, 2, 3)
        np.testing.assert_allclose(th2[p], mn + L @ z, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ll2, O.loglik(spec, y, th2, X=X), rtol=1e-13)
    # phi = 0 targets the prior: the prior as proposal is accepted everywhere
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    _, _, _, _, acc0, n0 = O.mutate_indep(spec, y, th, ll, lp, st, m0, np.diag(s0), 0.0, 7, 2, 4, X=X)
    assert n0 == P
    # a proposal off the posterior is not accepted everywhere
    _, _, _, _, _, n1 = O.mutate_indep(spec, y, th, ll, lp, st, mn + 0.05, L, 1.0, 7, 2, 3, X=X)
    assert n1 < P


def test_indep_kernel_leaves_posterior_invariant():
    """A proposal wider than and offset from the posterior still leaves the
    posterior invariant (detailed balance needs the q correction)."""
    spec, X, y, _, mn, Vn, _ = _linreg_problem()
    rng = np.random.default_rng(32)
    P = 20000
    th = rng.multivariate_normal(mn, Vn, size=P)
    ll = O.loglik(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    L = np.linalg.cholesky(1.5 ** 2 * Vn)
    mbar = mn + 0.5 * np.sqrt(np.diag(Vn))
    st = np.zeros((P, 1))
    for it in range(4):
        th, ll, lp, st, acc, nacc = O.mutate_indep(spec, y, th, ll, lp, st, mbar, L, 1.0, 9, 1, it, X=X)
    assert 0.2 < nacc / P < 0.9
    se = np.sqrt(np.diag(Vn) / P) * 2
    assert np.all(np.abs(th.mean(axis=0) - mn) < 4 * se)
    np.testing.assert_allclose(np.cov(th.T), Vn, rtol=0.06, atol=0.03 * np.abs(Vn).max())


@pytest.mark.parametrize("tempering", [0, 1])
def test_full_run_independent_sampler_matches_closed_form(tempering):
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 512
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=43)
    r = O.smc_run(spec, y, th0, J, N, X=X, tempering=tempering, mutation=O.INDEP, seed=17)
    assert r["status"] == 0
    assert abs(r["log_ml"] - lml) < 4.0 * r["log_ml_nse"] + 0.02
    for i in range(3):
        mean, sd, nse, rne = O.moment(r["theta"][:, i], J, N)
        assert abs(mean - mn[i]) < 4 * nse + 1e-4
    # a recorded design holds no proposal means: the independent sampler refuses it
    assert O.smc_run(spec, y, th0, J, N, X=X, mutation=O.INDEP, record=True)["status"] == -4


# ------------------------------------------ log score and PIT (Section 4.1)
def _linreg_prefix_lml(X, y, m0, s0, t):
    V0 = np.diag(s0 ** 2)
    return stats.multivariate_normal(X[:t] @ m0, np.eye(t) + X[:t] @ V0 @ X[:t].T).logpdf(y[:t])


def test_log_score_matches_closed_form():
    """log p(y_{b+1:T} | y_{1:b}) = log p(y_{1:T}) - log p(y_{1:b}) for the
    conjugate regression; the run ends a cycle at b."""
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    b = 20
    exact = lml - _linreg_prefix_lml(X, y, m0, s0, b)
    J, N = 8, 512
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=51)
    r = O.smc_run(spec, y, th0, J, N, X=X, tempering=0, burnin=b, seed=19)
    assert r["status"] == 0 and b in r["t"]
    assert abs(r["log_score"] - exact) < 4 * r["log_score_nse"] + 0.02, (r["log_score"], exact)
    assert abs(r["log_ml"] - lml) < 4 * r["log_ml_nse"] + 0.02
    # the log score is the later factor of the log ML, and nothing without a burn-in
    assert r["log_score"] > r["log_ml"]
    r0 = O.smc_run(spec, y, th0, J, N, X=X, tempering=0, seed=19)
    assert math.isnan(r0["log_score"])
    assert O.smc_run(spec, y, th0, J, N, X=X, tempering=1, burnin=b)["status"] == -5


def test_pit_matches_closed_form_predictive_cdf():
    """PIT of y_s: the weighted share of simulated Y_s <= y_s tracks the exact
    predictive CDF Phi((y_s - x_s'm_{s-1}) / (sigma^2 + x_s'V_{s-1}x_s)^{1/2})."""
    spec, X, y, lml, mn, Vn, (m0, s0) = _linreg_problem()
    J, N = 8, 1024
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=52)
    r = O.smc_run(spec, y, th0, J, N, X=X, tempering=0, pit=True, seed=23)
    assert r["status"] == 0
    Vinv, b = np.diag(1 / s0 ** 2), np.diag(1 / s0 ** 2) @ m0
    exact = np.zeros(len(y))
    for s in range(len(y)):
        V = np.linalg.inv(Vinv)
        m = V @ b
        x = X[s]
        exact[s] = stats.norm.cdf((y[s] - x @ m) / math.sqrt(1.0 + x @ V @ x))
        Vinv = Vinv + np.outer(x, x)
        b = b + x * y[s]
    err = np.abs(r["pit"] - exact)
    assert err.max() < 0.08 and err.mean() < 0.02, (err.max(), err.mean())
    # under the true model the transforms are uniform on (0, 1)
    assert stats.kstest(exact, "uniform").pvalue > 1e-3


def test_pit_shock_draws_the_mixture():
    """The simulated standardized shock of an EGARCH particle follows its
    normal mixture (Kolmogorov-Smirnov against the mixture CDF)."""
    spec = O.ModelSpec(K=1, I=2, gamma=True)
    mean, sd, lo = O.table1_prior(1, 2)
    th = I.draw_prior(mean, sd, lo, 1, seed=4)[0]
    par = O.egarch_transform(1, 2, True, th)
    assert min(par["p"]) < 0.4 and abs(par["mu"][0]) > 0.05   # an uneven, shifted mixture
    e = np.array([O.pit_shock(spec, th, 9, n, 3) for n in range(20000)])
    p, mu, sg = par["p"][:2], par["mu"][:2], par["sig"][:2]
    cdf = lambda x: sum(p[i] * stats.norm.cdf((x - mu[i]) / sg[i]) for i in range(2))
    assert stats.kstest(e, cdf).pvalue > 1e-3
    assert abs(e.mean()) < 0.03 and abs(e.var() - 1.0) < 0.05      # unit-variance mixture
    spec1 = O.ModelSpec(K=1, I=1, gamma=False)
    e1 = np.array([O.pit_shock(spec1, np.zeros(spec1.d), 9, n, 3) for n in range(20000)])
    assert stats.kstest(e1, "norm").pvalue > 1e-3


# ------------------------------------------------- prior draws (Table 1)
def test_prior_draws_follow_table1():
    """Philox prior draws: untruncated components are N(m, s^2) (KS), the
    truncated theta_8 components follow the truncated normal above -3 (KS),
    and a seed reproduces its draws while another seed changes them."""
    spec = O.ModelSpec(K=2, I=2, gamma=True)
    mean, sd, lo = O.table1_prior(2, 2)
    th = O.draw_prior(spec, 7, 20000)
    assert th.shape == (20000, spec.d)
    for i in range(spec.d):
        if np.isfinite(lo[i]):
            a = (lo[i] - mean[i]) / sd[i]
            assert th[:, i].min() >= lo[i]
            assert stats.kstest(th[:, i], stats.truncnorm(a, np.inf, loc=mean[i], scale=sd[i]).cdf).pvalue > 1e-3
        else:
            assert stats.kstest((th[:, i] - mean[i]) / sd[i], "norm").pvalue > 1e-3
    assert np.array_equal(th, O.draw_prior(spec, 7, 20000))
    assert not np.array_equal(th[:10], O.draw_prior(spec, 8, 10))
    # components are independent draws: no correlation between neighbours
    c = np.corrcoef(th[:, 0], th[:, 1])[0, 1]
    assert abs(c) < 0.03
