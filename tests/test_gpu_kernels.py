"""GPU parity of each kernel of the path against the FP64 oracle, through the
C ABI, on seeded inputs spanning several blocks/chunks with ragged tails.

Tolerances: log likelihood 1e-9 relative in FP64 and 1e-6 relative in FP32
(posterior-like particles; the FP32 contract is 1e-4);
resampling indices bit-exact given identical weights; estimators 1e-12."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1304_4334_gb300 import inputs as I
from tests.gpu_util import dev, egarch_truth, host, particles, soa, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch_cuda()
    from paper_1304_4334_gb300 import build
    build.build()
    from paper_1304_4334_gb300 import smc
    return smc


SHAPES = [(1, 1, False), (1, 1, True), (2, 1, True), (2, 2, True), (3, 4, True), (4, 3, False)]


def _loglik_case(S, K, I_, gamma, T, P, precision, seed, frac_prior=0.0):
    torch = torch_cuda()
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=seed)
    spec = O.ModelSpec(K=K, I=I_, gamma=gamma)
    prior = O.table1_prior(K, I_, gamma)
    th = particles(spec.d, truth, K, I_, gamma, P, seed + 7, prior=prior, frac_prior=frac_prior)
    ll_o, st_o = O.loglik(spec, y, th, with_state=True, nthreads=4)
    lp_o = O.logprior(spec, th)
    m = S.model_egarch(K, I_, gamma)
    obs = dev(y, torch.float32 if precision == S.FP32 else torch.float64)
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(ll)
    st = torch.empty((K + 1, P), dtype=torch.float64, device="cuda")
    S.loglik(m, precision, obs, soa(th), ll, lp, st)
    torch.cuda.synchronize()
    return ll_o, st_o, lp_o, host(ll), host(st).T, host(lp)


@pytest.mark.parametrize("K,I_", [(3, 4), (2, 3), (1, 4)])
def test_loglik_fp32_tail_observations_match_oracle(S, K, I_):
    """Outlying observations push every mixture component of many particles
    far into its tail: every 13th shock scaled by 10 to 60 and a run of 40
    shocks scaled by 5 (mixture sums far below their peak, observation after
    observation).  For posterior-like particles the FP32 recursion's log
    likelihood still matches the FP64 oracle; a mishandled tail would move it
    by tens of nats.  (Prior draws are left out here: with such shocks some of
    them reach volatilities of 2^1000 and beyond, where FP32 and FP64
    underflow at different points.)"""
    torch = torch_cuda()
    truth = egarch_truth(K, I_)
    T, P = 777, 400
    y = I.simulate_egarch(truth, T, seed=41)
    y[::13] *= np.linspace(10.0, 60.0, len(y[::13]))
    y[300:340] *= 5.0
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    prior = O.table1_prior(K, I_, True)
    th = particles(spec.d, truth, K, I_, True, P, 43, prior=prior, frac_prior=0.0)
    ll_o = O.loglik(spec, y, th, nthreads=4)
    m = S.model_egarch(K, I_, True)
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    S.loglik(m, S.FP32, dev(y, torch.float32), soa(th), ll, None, None)
    ll = host(ll)
    fin = np.isfinite(ll_o) & (ll_o > -1e7)
    assert fin.sum() >= P - 2 and np.all(np.isfinite(ll[fin]))
    err = np.abs(ll[fin] - ll_o[fin]) / np.abs(ll_o[fin])
    assert np.quantile(err, 0.99) <= 1e-5 and err.max() <= 1e-4, (np.quantile(err, 0.99), err.max())


@pytest.mark.parametrize("K,I_,gamma", SHAPES)
@pytest.mark.parametrize("T,P", [(1, 5), (37, 129), (1037, 300)])
def test_loglik_fp64_matches_oracle(S, K, I_, gamma, T, P):
    ll_o, st_o, lp_o, ll, st, lp = _loglik_case(S, K, I_, gamma, T, P, S.FP64, seed=3 + T)
    np.testing.assert_allclose(ll, ll_o, rtol=1e-9, atol=0)
    np.testing.assert_allclose(st, st_o, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(lp, lp_o, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("K,I_,gamma", SHAPES)
@pytest.mark.parametrize("T,P", [(1, 5), (37, 129), (3089, 300)])
def test_loglik_fp32_matches_oracle(S, K, I_, gamma, T, P):
    """FP32 recursion with FP64 accumulation, posterior-like particles: 1e-6
    relative (1e-7 measured; the stated FP32 tolerance is 1e-4)."""
    ll_o, st_o, lp_o, ll, st, lp = _loglik_case(S, K, I_, gamma, T, P, S.FP32, seed=5 + T)
    np.testing.assert_allclose(ll, ll_o, rtol=1e-6, atol=1e-6)
    # end state: eps_T and v_kT carry the FP32 recursion's rounding
    np.testing.assert_allclose(st, st_o, rtol=2e-3, atol=2e-3)
    np.testing.assert_allclose(lp, lp_o, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_loglik_prior_draws(S, precision):
    """Raw prior draws reach extreme volatility dynamics.  FP64 must match to
    1e-9 relative.  The FP32 likelihood kernel carries 1 - alpha_k itself
    (alpha close to 1 would lose it in FP32 rounding), which leaves the
    draws whose recursion amplifies any rounding: a large beta_k feeds each
    shock's error back into the next volatility, and a likelihood that is a
    small difference of large terms (|sum_t l_t| << sum_t |l_t|) shows its
    absolute error as a large relative one.  The bound for raw prior draws is
    therefore 99% of draws within 1e-4 relative and every draw within 1e-3 of
    sum_t |l_t|; the measured figures are printed.
    Where the oracle value is below -1e7 (a weight of zero at any precision)
    FP32 may saturate to -inf."""
    prec = S.FP64 if precision == "fp64" else S.FP32
    K, I_, gamma, T = 2, 2, True, 800
    ll_o, _, _, ll, _, _ = _loglik_case(S, K, I_, gamma, T, 1000, prec, seed=41, frac_prior=1.0)
    sane = ll_o > -1e7
    assert sane.mean() > 0.2
    if prec == S.FP64:
        np.testing.assert_allclose(ll[sane], ll_o[sane], rtol=1e-9)
    else:
        truth = egarch_truth(K, I_)
        y = I.simulate_egarch(truth, T, seed=41)
        spec = O.ModelSpec(K=K, I=I_, gamma=gamma)
        th = particles(spec.d, truth, K, I_, gamma, 1000, 48, prior=O.table1_prior(K, I_, gamma),
                       frac_prior=1.0)
        mag = np.array([np.abs(O.loglik_terms(spec, y, th[n])).sum() for n in range(1000)])
        err = np.abs(ll - ll_o)
        rel = err[sane] / np.abs(ll_o[sane])
        print(f"FP32 raw prior draws: max rel {rel.max():.2e}, median {np.median(rel):.2e}, "
              f"share <= 1e-4 {(rel <= 1e-4).mean():.4f}, max err / sum|l_t| {(err[sane] / mag[sane]).max():.2e}")
        assert np.all(err[sane] <= 1e-3 * mag[sane]), (err[sane] / mag[sane]).max()
        within = err[sane] <= 1e-4 * np.abs(ll_o[sane]) + 1e-4
        assert within.mean() >= 0.99, within.mean()
    assert np.all(ll[~sane] < -1e6)


def test_loglik_fixed_parameters_and_eps0_reading(S):
    torch = torch_cuda()
    truth = egarch_truth(1, 1)
    y = I.simulate_egarch(truth, 300, seed=2)
    th_true = I.theta_of_truth(truth)
    grid = np.linspace(-6, -3.5, 101)[:, None]
    spec = O.ModelSpec(K=1, I=1, gamma=True, free_idx=[1], theta_fixed=th_true)
    m = S.model_egarch(1, 1, True, free_idx=[1], theta_fixed=th_true)
    ll = torch.empty(101, dtype=torch.float64, device="cuda")
    S.loglik(m, S.FP64, dev(y), soa(grid), ll)
    np.testing.assert_allclose(host(ll), O.loglik(spec, y, grid), rtol=1e-9)
    spec0 = O.ModelSpec(K=1, I=1, gamma=True, eps0_zero=True)
    m0 = S.model_egarch(1, 1, True, eps0_zero=True)
    th = I.posterior_cloud(th_true, 64, 0.05, 3)
    S.loglik(m0, S.FP64, dev(y), soa(th), ll[:64])
    np.testing.assert_allclose(host(ll[:64]), O.loglik(spec0, y, th), rtol=1e-9)


def test_loglik_linreg(S):
    torch = torch_cuda()
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(301, beta, 0.7, seed=4)
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=0.7, prior_mean=np.zeros(3), prior_sd=np.full(3, 2.0))
    m = S.model_linreg(3, 0.7, np.zeros(3), np.full(3, 2.0))
    W = S.linreg_width(3)
    rec = np.zeros((301, W))
    rec[:, :3] = X
    rec[:, 3] = y
    th = beta + 0.1 * np.random.default_rng(1).standard_normal((500, 3))
    ll = torch.empty(500, dtype=torch.float64, device="cuda")
    lp = torch.empty_like(ll)
    S.loglik(m, S.FP64, dev(rec.reshape(-1)).reshape(301, W), soa(th), ll, lp)
    np.testing.assert_allclose(host(ll), O.loglik(spec, y, th, X=X), rtol=1e-11)
    np.testing.assert_allclose(host(lp), O.logprior(spec, th), rtol=1e-13)


# --------------------------------------------------------------------- M phase
def _oracle_log_alpha(spec, y, th, ll, lp, Lm, phi, seed, cycle, it):
    P, d = th.shape
    la = np.zeros(P)
    lu = np.zeros(P)
    for n in range(P):
        z = O.philox_normals(seed, n, it, cycle, d)
        prop = th[n] + Lm @ z
        lpn = O.logprior(spec, prop)[0]
        lln = O.loglik(spec, y, prop)[0] if lpn > -np.inf else -np.inf
        la[n] = (lpn + phi * lln) - (lp[n] + phi * ll[n])
        lu[n] = O.philox_log_uniform(seed, n, it, cycle)
    return la, lu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mutate_step_matches_oracle(S, precision):
    torch = torch_cuda()
    prec = S.FP64 if precision == "fp64" else S.FP32
    K, I_, T, P = 2, 2, 300, 1111
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=9)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 12)
    ll, st = O.loglik(spec, y, th, with_state=True, nthreads=4)
    lp = O.logprior(spec, th)
    _, V = O.mean_cov(th)
    Lm, _ = O.cholesky(0.3 ** 2 * V)
    phi, seed, cycle, it = 0.7, 77, 3, 2
    th_o, ll_o, lp_o, st_o, acc_o, nacc_o = O.mutate_rw(spec, y, th, ll, lp, st, Lm, phi, seed, cycle, it,
                                                        nthreads=4)
    m = S.model_egarch(K, I_, True)
    obs = dev(y, torch.float32 if prec == S.FP32 else torch.float64)
    tg, llg, lpg = soa(th), dev(ll), dev(lp)
    stg = soa(st)
    nacc = S.mutate_rw(m, prec, obs, tg, llg, lpg, stg, dev(Lm), phi, seed, cycle, it)
    th_g, ll_g, lp_g, st_g = host(tg).T, host(llg), host(lpg), host(stg).T
    acc_g = np.any(th_g != th, axis=1)
    assert nacc == acc_g.sum()
    diff = acc_g != acc_o.astype(bool)
    if diff.any():   # only where the decision is within rounding of the threshold
        idx = np.nonzero(diff)[0]
        la_all, lu_all = _oracle_log_alpha(spec, y, th, ll, lp, Lm, phi, seed, cycle, it)
        margin = np.abs(la_all[idx] - lu_all[idx])
        # the decision may differ only within the rounding of log alpha: FP64
        # ~1e-12; FP32 ~1e-6 of the log-likelihood magnitude (10x margin)
        scale = phi * (np.abs(ll[idx]) + np.abs(ll_o[idx]))
        bound = 1e-8 if prec == S.FP64 else 1e-5 * scale + 1e-6
        assert np.all(margin < bound), (margin, bound)
        assert diff.sum() <= max(2, P // 100)
    same = ~diff
    tol = 1e-9 if prec == S.FP64 else 1e-4
    np.testing.assert_allclose(th_g[same], th_o[same], rtol=tol, atol=1e-6 if prec == S.FP32 else 1e-12)
    np.testing.assert_allclose(ll_g[same], ll_o[same], rtol=tol)
    np.testing.assert_allclose(lp_g[same], lp_o[same], rtol=tol, atol=tol)
    np.testing.assert_allclose(st_g[same], st_o[same], rtol=2e-3 if prec == S.FP32 else 1e-9,
                               atol=2e-3 if prec == S.FP32 else 1e-12)
    assert 0.05 < nacc / P < 0.95


def _oracle_log_alpha_indep(spec, y, th, ll, lp, mbar, Lm, phi, seed, cycle, it):
    """log alpha of the independent sampler for every particle, by the oracle's
    likelihood and a triangular solve, for judging decisions near the threshold."""
    from scipy.linalg import solve_triangular
    P, d = th.shape
    la = np.zeros(P)
    lu = np.zeros(P)
    for n in range(P):
        z = O.philox_normals(seed, n, it, cycle, d)
        prop = mbar + Lm @ z
        lpn = O.logprior(spec, prop)[0]
        lln = O.loglik(spec, y, prop)[0] if lpn > -np.inf else -np.inf
        u = solve_triangular(Lm, th[n] - mbar, lower=True)
        la[n] = (lpn + phi * lln) - (lp[n] + phi * ll[n]) - 0.5 * u @ u + 0.5 * z @ z
        lu[n] = O.philox_log_uniform(seed, n, it, cycle)
    return la, lu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mutate_indep_step_matches_oracle(S, precision):
    """Independent Gaussian sampler (Section 3.3): same proposals at
    mean + L z, same log q correction and decisions as the oracle."""
    torch = torch_cuda()
    prec = S.FP64 if precision == "fp64" else S.FP32
    K, I_, T, P = 2, 2, 300, 1111
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=19)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 13)
    ll, st = O.loglik(spec, y, th, with_state=True, nthreads=4)
    lp = O.logprior(spec, th)
    mbar, V = O.mean_cov(th)
    Lm, _ = O.cholesky(V)
    phi, seed, cycle, it = 0.05, 78, 4, 1
    th_o, ll_o, lp_o, st_o, acc_o, nacc_o = O.mutate_indep(spec, y, th, ll, lp, st, mbar, Lm, phi, seed,
                                                           cycle, it, nthreads=4)
    m = S.model_egarch(K, I_, True)
    obs = dev(y, torch.float32 if prec == S.FP32 else torch.float64)
    tg, llg, lpg, stg = soa(th), dev(ll), dev(lp), soa(st)
    nacc = S.mutate_indep(m, prec, obs, tg, llg, lpg, stg, dev(mbar), dev(Lm), phi, seed, cycle, it)
    th_g, ll_g, lp_g, st_g = host(tg).T, host(llg), host(lpg), host(stg).T
    acc_g = np.any(th_g != th, axis=1)
    assert nacc == acc_g.sum()
    diff = acc_g != acc_o.astype(bool)
    if diff.any():
        idx = np.nonzero(diff)[0]
        la_all, lu_all = _oracle_log_alpha_indep(spec, y, th, ll, lp, mbar, Lm, phi, seed, cycle, it)
        margin = np.abs(la_all[idx] - lu_all[idx])
        scale = phi * (np.abs(ll[idx]) + np.abs(ll_o[idx]))
        bound = 1e-8 if prec == S.FP64 else 1e-5 * scale + 1e-5
        assert np.all(margin < bound), (margin, bound)
        assert diff.sum() <= max(2, P // 100)
    same = ~diff
    tol = 1e-9 if prec == S.FP64 else 1e-4
    np.testing.assert_allclose(th_g[same], th_o[same], rtol=tol, atol=1e-6 if prec == S.FP32 else 1e-12)
    np.testing.assert_allclose(ll_g[same], ll_o[same], rtol=tol)
    np.testing.assert_allclose(lp_g[same], lp_o[same], rtol=tol, atol=tol)
    np.testing.assert_allclose(st_g[same], st_o[same], rtol=2e-3 if prec == S.FP32 else 1e-9,
                               atol=2e-3 if prec == S.FP32 else 1e-12)
    assert 0.02 < nacc / P < 0.98


def test_mutate_indep_exact_posterior_accepts_all(S):
    """Conjugate regression with q the exact posterior: every proposal is
    accepted at mean + L z, as the oracle's pin states."""
    torch = torch_cuda()
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(60, beta, 1.0, seed=3)
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    Vn = np.linalg.inv(np.diag(1 / s0 ** 2) + X.T @ X)
    mn = Vn @ (X.T @ y)
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=1.0, prior_mean=m0, prior_sd=s0)
    m = S.model_linreg(3, 1.0, m0, s0)
    rec = np.zeros((60, S.linreg_width(3)))
    rec[:, :3] = X
    rec[:, 3] = y
    P = 2000
    th = np.random.default_rng(4).multivariate_normal(mn, 3 * Vn, size=P)
    ll = O.loglik(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    Lm = np.linalg.cholesky(Vn)
    tg, llg, lpg = soa(th), dev(ll), dev(lp)
    nacc = S.mutate_indep(m, S.FP64, dev(rec), tg, llg, lpg, None, dev(mn), dev(Lm), 1.0, 3, 2, 5)
    assert nacc == P
    th_o, ll_o, *_ = O.mutate_indep(spec, y, th, ll, lp, np.zeros((P, 1)), mn, Lm, 1.0, 3, 2, 5, X=X)
    np.testing.assert_allclose(host(tg).T, th_o, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(host(llg), ll_o, rtol=1e-11)


def test_mutate_linreg_matches_oracle(S):
    torch = torch_cuda()
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(200, beta, 1.0, seed=6)
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=1.0, prior_mean=np.zeros(3), prior_sd=np.full(3, 2.0))
    m = S.model_linreg(3, 1.0, np.zeros(3), np.full(3, 2.0))
    rec = np.zeros((200, S.linreg_width(3)))
    rec[:, :3] = X
    rec[:, 3] = y
    P = 777
    th = beta + 0.1 * np.random.default_rng(3).standard_normal((P, 3))
    ll = O.loglik(spec, y, th, X=X)
    lp = O.logprior(spec, th)
    Lm = np.linalg.cholesky(0.01 * np.eye(3))
    th_o, ll_o, lp_o, _, acc_o, nacc_o = O.mutate_rw(spec, y, th, ll, lp, np.zeros((P, 1)), Lm, 1.0, 5, 1, 0, X=X)
    tg, llg, lpg = soa(th), dev(ll), dev(lp)
    nacc = S.mutate_rw(m, S.FP64, dev(rec), tg, llg, lpg, None, dev(Lm), 1.0, 5, 1, 0)
    assert nacc == nacc_o
    np.testing.assert_allclose(host(tg).T, th_o, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(host(llg), ll_o, rtol=1e-11)


# ------------------------------------------------------------- covariance
@pytest.mark.parametrize("d,P", [(4, 1024), (14, 65536 + 37), (23, 5000), (1, 300)])
def test_cov_chol_matches_oracle_and_numpy(S, d, P):
    torch = torch_cuda()
    rng = np.random.default_rng(d)
    A = rng.normal(size=(d, d)) * 0.1
    th = rng.normal(size=(P, d)) @ A + rng.normal(0, 3, d)
    mean = torch.empty(d, dtype=torch.float64, device="cuda")
    cov = torch.empty((d, d), dtype=torch.float64, device="cuda")
    L = torch.empty((d, d), dtype=torch.float64, device="cuda")
    S.cov_chol(soa(th), 7, mean, cov, L)
    m_o, c_o = O.mean_cov(th) if P <= 5000 else (th.mean(0), np.cov(th.T))
    c_o = np.atleast_2d(c_o)
    # products are summed in FP32 within 64-particle tiles (see the kernel):
    # about 1e-6 relative, far inside what a proposal scale needs
    sdv = np.sqrt(np.diag(c_o))
    np.testing.assert_allclose(host(mean), m_o, rtol=0, atol=1e-6 * sdv.max())
    np.testing.assert_allclose(host(cov), c_o, rtol=1e-5, atol=1e-6 * np.abs(c_o).max())
    Lw = np.linalg.cholesky(0.49 * c_o)
    np.testing.assert_allclose(host(L), Lw, rtol=1e-4, atol=1e-5 * np.abs(Lw).max())


def test_cov_chol_rank_deficient(S):
    torch = torch_cuda()
    rng = np.random.default_rng(0)
    x = rng.normal(size=(400, 1))
    th = np.hstack([x, 2 * x, rng.normal(size=(400, 1))])
    L = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    S.cov_chol(soa(th), 10, None, None, L)
    Lo, z = O.cholesky(np.cov(th.T))
    Lg = host(L)
    assert abs(Lg[1, 1]) < 1e-3 and z == 1
    np.testing.assert_allclose(Lg @ Lg.T, np.cov(th.T), atol=1e-5)


# ------------------------------------------------------------------ C phase
# Each block keeps its range of particles in shared memory up to 16,384 of
# them (2,490,368 particles on 152 SMs); 3,000,017 go through global scratch
# staged once per pass, 7,500,001 in two stages per pass (49,344 per block
# against 49,152 staged at a time).  33 leave most warps of the only block
# empty.
@pytest.mark.parametrize("P,phi,spread", [(65536, 0.0, 30.0), (1024, 0.3, 5.0), (4096, 0.9, 200.0),
                                          (400037, 0.2, 50.0), (33, 0.0, 3.0), (3000017, 0.1, 40.0),
                                          (7500001, 0.0, 60.0)])
def test_power_search_matches_oracle(S, P, phi, spread):
    rng = np.random.default_rng(P)
    ll = -16000 + spread * rng.standard_normal(P)
    ll[:3] = -np.inf
    d_o, r_o = O.power_search(ll, phi, 0.5)
    d_g, r_g = S.power_search(dev(ll), phi, 0.5, passes=6)
    if d_o < 1 - phi:
        assert d_g == pytest.approx(d_o, rel=1e-4)
        if P <= 8192:
            # the search compares RSS with FP32 weights, so the FP64 RSS at the
            # chosen power sits within about 1e-6 of D1
            assert r_g == pytest.approx(0.5, abs=1e-5) and r_g < 0.5 + 1e-6
    else:
        assert d_g == 1 - phi


def test_power_search_takes_remaining_power_when_flat(S):
    ll = np.full(2048, -1234.5)
    d_g, r_g = S.power_search(dev(ll), 0.25, 0.5)
    assert d_g == 0.75 and r_g == pytest.approx(1.0, rel=1e-12)


# ------------------------------------------------------------------ S phase
@pytest.mark.parametrize("J,N,resid", [(64, 1024, True), (3, 1000, True), (5, 8192, True),
                                       (7, 333, False), (2, 1, True), (16, 4096, False)])
def test_resample_bit_exact(S, J, N, resid):
    torch = torch_cuda()
    rng = np.random.default_rng(J * N)
    w = rng.gamma(0.3, size=J * N)
    w[rng.random(J * N) < 0.1] = 0.0
    if N > 1:
        w.reshape(J, N)[:, 0] += 1e-3
    idx_o = O.resample(w, J, N, resid=resid, seed=9, cycle=4)
    idx = torch.empty(J * N, dtype=torch.int32, device="cuda")
    S.resample(dev(w), J, N, idx, S.RESIDUAL if resid else S.MULTINOMIAL, seed=9, cycle=4)
    assert np.array_equal(host(idx).reshape(J, N), idx_o)


@pytest.mark.parametrize("J,N,scheme", [(64, 1024, 2), (64, 1024, 3), (3, 1000, 2), (5, 8192, 3),
                                         (7, 333, 3), (2, 1, 2)])
def test_stratified_systematic_bit_exact(S, J, N, scheme):
    torch = torch_cuda()
    rng = np.random.default_rng(J * N + scheme)
    w = rng.gamma(0.3, size=J * N)
    w[rng.random(J * N) < 0.1] = 0.0
    w.reshape(J, N)[:, 0] += 1e-3
    idx_o = O.resample_scheme(w, J, N, scheme, seed=5, cycle=2)
    idx = torch.empty(J * N, dtype=torch.int32, device="cuda")
    S.resample(dev(w), J, N, idx, scheme, seed=5, cycle=2)
    assert np.array_equal(host(idx).reshape(J, N), idx_o)


def _log_weight_cases(J, N, rng, kind):
    """Log weights of the shapes the S phase meets: tempered log likelihoods
    (dphi l_n, wide spread), data-tempering increments (narrow), weights
    spanning the fixed point's whole range, dead particles and exact ties."""
    if kind == "power":
        lw = 1e-3 * (-30000.0 + 4000.0 * rng.standard_normal(J * N))
    elif kind == "data":
        lw = 0.3 * rng.standard_normal(J * N) - 2.0
    else:
        lw = -rng.uniform(0.0, 70.0, J * N)
        lw[rng.random(J * N) < 0.05] = -np.inf
        g = lw.reshape(J, N)
        g[:, 0] = 0.0
        if N > 3:
            g[:, 1] = 0.0                      # ties at the maximum
            g[:, 2] = -2.0 ** -52              # exp(x) just below one
            g[:, 3] = -1e-20                   # exp(x) rounds to one
    return lw


@pytest.mark.parametrize("J,N,scheme,kind", [(64, 1024, 0, "power"), (128, 8192, 0, "power"),
                                              (5, 8192, 1, "data"), (7, 333, 0, "wide"),
                                              (16, 4096, 2, "wide"), (3, 1000, 3, "data"),
                                              (2, 1, 0, "wide"), (33, 2048, 0, "wide")])
def test_resample_from_log_weights_bit_exact(S, J, N, scheme, kind):
    """The in-run S phase (weights from log weights by the fixed-point
    exponential) selects exactly the oracle's indices for the FP64 weights
    exp(lw - max), and its log wbar_j is the group's log mean weight."""
    torch = torch_cuda()
    rng = np.random.default_rng(J * N + scheme)
    lw = _log_weight_cases(J, N, rng, kind)
    g = lw.reshape(J, N)
    w = np.exp(g - g.max(axis=1, keepdims=True)).reshape(-1)
    if scheme <= 1:
        idx_o = O.resample(w, J, N, resid=scheme == 0, seed=11, cycle=7)
    else:
        idx_o = O.resample_scheme(w, J, N, scheme, seed=11, cycle=7)
    idx = torch.empty(J * N, dtype=torch.int32, device="cuda")
    lwbar = S.resample_logw(dev(lw), J, N, idx, scheme, seed=11, cycle=7)
    assert np.array_equal(host(idx).reshape(J, N), idx_o)
    mx = g.max(axis=1)
    want = mx + np.log(np.exp(g - mx[:, None]).sum(axis=1) / N)
    err = np.abs(lwbar - want) / np.maximum(1.0, np.abs(want))
    assert err.max() <= 1e-13, err.max()


def test_resample_from_log_weights_degenerate(S):
    torch = torch_cuda()
    lw = np.zeros(2 * 64)
    lw[64:] = -np.inf
    idx = torch.empty(128, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SMCError) as e:
        S.resample_logw(dev(lw), 2, 64, idx)
    assert e.value.status == S.EDEGENERATE
    assert np.array_equal(host(idx)[64:], np.arange(64))


def test_resample_dominant_and_degenerate(S):
    torch = torch_cuda()
    N = 8192
    w = np.full(N, 1e-3)
    w[5] = 1.0
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    S.resample(dev(w), 1, N, idx, seed=2, cycle=3)
    assert np.array_equal(host(idx), O.resample(w, 1, N, seed=2, cycle=3)[0])
    w = np.zeros(2 * 64)
    w[70] = 1.0
    idx = torch.empty(128, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SMCError) as e:
        S.resample(dev(w), 2, 64, idx)
    assert e.value.status == S.EDEGENERATE


# -------------------------------------------------------------- estimators
def test_group_moments_and_ml_match_oracle(S):
    rng = np.random.default_rng(5)
    J, N = 64, 1024
    g = rng.normal(size=(3, J * N)) * np.array([[1.0], [3.0], [0.01]]) + np.array([[5.0], [-2.0], [0.1]])
    out = S.group_moments(dev(g), J, N)
    for f in range(3):
        want = O.moment(g[f], J, N)
        np.testing.assert_allclose(out[f], want, rtol=1e-11)
    a = rng.normal(-12000, 0.05, J)
    x, s = S.ml_from_groups(dev(a))
    xo, so = O.log_ml(a)
    assert x == pytest.approx(xo, rel=1e-14) and s == pytest.approx(so, rel=1e-10)


def test_bounded_wait_times_out_and_the_context_survives(S):
    """Failure detection without a fault: the library's bounded mbarrier wait
    on a barrier nothing completes returns SMC_ETIMEOUT after its limit, the
    same wait on a completed barrier returns OK, and device work still runs
    afterwards."""
    import time
    torch = torch_cuda()
    t0 = time.perf_counter()
    assert S.wait_selftest(20_000_000, False) == S.ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert S.wait_selftest(20_000_000, True) == S.OK
    K, I_, T, P = 1, 1, 64, 40
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=3)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 4)
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    S.loglik(S.model_egarch(K, I_, True), S.FP64, dev(y), soa(th), ll)
    np.testing.assert_allclose(host(ll), O.loglik(spec, y, th), rtol=1e-9)


def test_prior_draws_match_the_oracle(S):
    """Device prior draws (Table 1, Philox counters, truncation by rejection)
    equal the oracle's to rounding, for EGARCH(2,2) and the regression."""
    torch = torch_cuda()
    for K, I_ in [(2, 2), (3, 4), (1, 1)]:
        spec = O.ModelSpec(K=K, I=I_, gamma=True)
        m = S.model_egarch(K, I_, True)
        th = host(S.draw_prior(m, 11, 5003)).T
        th_o = O.draw_prior(spec, 11, 5003)
        np.testing.assert_allclose(th, th_o, rtol=1e-12, atol=1e-13)
        mean, sd, lo = O.table1_prior(K, I_)
        assert np.all(th >= lo)
