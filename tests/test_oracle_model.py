"""Pins for the oracle's model code (Section 5.1, Table 1, Section 5.2).

Each check compares the oracle with something other than itself: the Table 1
fixture, library densities (scipy), the forward simulator of the
data-generating process (inverted exactly by the likelihood recursion),
numerical quadrature, invariances the model must have, or finite differences."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_1304_4334_gb300 import inputs as I
from tests.golden_io import table1_vector

SHAPES = [(1, 1, False), (1, 1, True), (2, 2, True), (3, 4, True), (2, 3, False)]


@pytest.mark.parametrize("K,Imix,gamma", SHAPES)
def test_table1_prior_matches_fixture(K, Imix, gamma):
    want = table1_vector(K, Imix, gamma)
    got = O.table1_prior(K, Imix, gamma)
    for w, g in zip(want, got):
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-15)
    assert O.egarch_dim(K, Imix, gamma) == 2 + 2 * K + (K if gamma else 0) + (3 * Imix if Imix >= 2 else 0)


@pytest.mark.parametrize("K,Imix", [(2, 2), (3, 4), (1, 3)])
def test_mixture_normalisation_invariants(K, Imix):
    # (EGARCH_normalization): sum p mu = 0 and sum p (mu^2 + sigma^2) = 1
    rng = np.random.default_rng(1)
    d = O.egarch_dim(K, Imix, True)
    for _ in range(50):
        th = rng.normal(0, 1.5, d)
        q = O.egarch_transform(K, Imix, True, th)
        assert abs(np.sum(q["p"]) - 1) < 1e-14
        assert abs(np.sum(q["p"] * q["mu"])) < 1e-13
        assert abs(np.sum(q["p"] * (q["mu"] ** 2 + q["sig"] ** 2)) - 1) < 1e-13
        assert np.all(np.abs(q["alpha"]) < 1) and np.all(q["beta"] > 0)


def test_transform_closed_form_two_components():
    # theta_6 = 0 gives p* = 1 each, so p = 1/2; mu* = +-a; sigma* = 1:
    # mu** = +-a, c = (a^2 + 1)^{-1/2}
    a = 0.7
    th = np.array([2.0, math.log(0.02), 0.3, -1.0, 0.1, 0.0, 0.0, a, -a, 0.0, 0.0])
    q = O.egarch_transform(1, 2, True, th)
    c = 1 / math.sqrt(a * a + 1)
    np.testing.assert_allclose(q["p"], [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(q["mu"], [c * a, -c * a], atol=1e-15)
    np.testing.assert_allclose(q["sig"], [c, c], atol=1e-15)
    assert q["mu_y"] == pytest.approx(0.002, abs=1e-18)
    assert q["sigma_y"] == pytest.approx(0.02, rel=1e-15)
    assert q["alpha"][0] == pytest.approx(math.tanh(0.3), rel=1e-15)
    assert q["beta"][0] == pytest.approx(math.exp(-1.0), rel=1e-15)


def test_logprior_matches_scipy_and_truncation():
    spec = O.ModelSpec(K=2, I=2, gamma=True)
    m, s, lo = O.table1_prior(2, 2, True)
    rng = np.random.default_rng(3)
    th = I.draw_prior(m, s, lo, 20, 5)
    want = stats.norm.logpdf(th, m, s).sum(axis=1)
    np.testing.assert_allclose(O.logprior(spec, th), want, rtol=1e-13)
    bad = th[0].copy()
    bad[-1] = -3.0001            # theta_8I below its truncation point
    assert O.logprior(spec, bad)[0] == -np.inf


TRUTHS = {
    "k1i1": I.EgarchTruth(0.0004, 0.012, (0.95,), (0.12,), (-0.06,)),
    "k2i2": I.WORKLOADS["egarch22_T5000"].truth,
    "k3i4": I.EgarchTruth(0.0002, 0.01, (0.97, 0.8, 0.4), (0.07, 0.1, 0.2), (-0.03, 0.02, -0.05),
                          *I.normalized_mixture((0.5, 0.2, 0.2, 0.1), (0.1, -0.2, 0.3, -0.4),
                                                (0.8, 1.2, 1.5, 3.0))),
}


@pytest.mark.parametrize("name", list(TRUTHS))
def test_loglik_inverts_the_simulator(name):
    """The recursion must recover the simulator's shocks eps_t and volatilities h_t
    exactly, and the likelihood must equal sum_t [log f_mix(eps_t) - log h_t] with
    f_mix built from scipy's normal density."""
    tr = TRUTHS[name]
    T = 400
    y, eps, h, v_T, _ = I.simulate_egarch(tr, T, seed=17, return_path=True)
    spec = O.ModelSpec(K=tr.K, I=tr.I, gamma=True)
    th = I.theta_of_truth(tr)
    q = O.egarch_transform(tr.K, tr.I, True, th)
    np.testing.assert_allclose(q["p"], tr.p, rtol=1e-12)
    np.testing.assert_allclose(q["sig"], tr.sig, rtol=1e-12)
    ll, st = O.loglik(spec, y, th, with_state=True)
    np.testing.assert_allclose(st[0, :tr.K], v_T, rtol=1e-9, atol=1e-12)
    assert st[0, tr.K] == pytest.approx(eps[-1], rel=1e-9)
    fmix = sum(p * stats.norm.pdf(eps, m, s) for p, m, s in zip(tr.p, tr.mu, tr.sig))
    want = np.sum(np.log(fmix) - np.log(h))
    assert ll[0] == pytest.approx(want, rel=1e-12)
    terms = O.loglik_terms(spec, y, th)
    np.testing.assert_allclose(terms, np.log(fmix) - np.log(h), rtol=1e-10, atol=1e-10)


def test_loglik_without_dynamics_is_iid_normal():
    # alpha = beta = gamma = 0 (beta = e^-60 is zero to double precision in
    # the recursion's output), I = 1: sum log N(y_t; mu_Y, sigma_Y^2).
    spec = O.ModelSpec(K=1, I=1, gamma=True)
    rng = np.random.default_rng(2)
    y = rng.normal(0, 0.01, 300)
    th = np.array([0.5, math.log(0.011), 0.0, -60.0, 0.0])
    want = stats.norm.logpdf(y, 0.5 / 1000, 0.011).sum()
    assert O.loglik(spec, y, th)[0] == pytest.approx(want, rel=1e-13)


def test_eps0_zero_reading_shifts_first_volatility():
    # with eps_0 = 0, v_k1 = -beta_k (2/pi)^{1/2}; h_1 = sigma_Y exp(v_11/2)
    spec = O.ModelSpec(K=1, I=1, gamma=True, eps0_zero=True)
    th = np.array([0.0, math.log(0.01), 0.5, math.log(0.2), 0.0])
    y = np.array([0.013])
    h1 = 0.01 * math.exp(-0.2 * math.sqrt(2 / math.pi) / 2)
    assert O.loglik(spec, y, th)[0] == pytest.approx(stats.norm.logpdf(0.013, 0, h1), rel=1e-13)


def test_predictive_density_integrates_to_one():
    tr = TRUTHS["k3i4"]
    spec = O.ModelSpec(K=3, I=4, gamma=True)
    th = I.theta_of_truth(tr)
    y = I.simulate_egarch(tr, 30, seed=4)
    base = O.loglik(spec, y[:29], th)[0]

    def dens(x):
        yy = y.copy()
        yy[29] = x
        return math.exp(O.loglik(spec, yy, th)[0] - base)

    mass, _ = integrate.quad(dens, -1.0, 1.0, limit=400, points=[tr.mu_y])
    assert mass == pytest.approx(1.0, abs=1e-8)


def test_permutation_invariance():
    spec = O.ModelSpec(K=3, I=4, gamma=True)
    rng = np.random.default_rng(9)
    th = I.theta_of_truth(TRUTHS["k3i4"]) + rng.normal(0, 0.1, 23)
    y = I.simulate_egarch(TRUTHS["k3i4"], 300, seed=5)
    base = O.loglik(spec, y, th)[0]
    K, Im = 3, 4
    fac = np.array([1, 2, 0])           # permute factors (theta_3k, theta_4k, theta_5k)
    t2 = th.copy()
    for blk in range(3):
        t2[2 + blk * K: 2 + (blk + 1) * K] = th[2 + blk * K: 2 + (blk + 1) * K][fac]
    assert O.loglik(spec, y, t2)[0] == pytest.approx(base, rel=1e-12)
    comp = np.array([3, 0, 2, 1])       # permute mixture components (theta_6i, 7i, 8i)
    t3 = th.copy()
    off = 2 + 3 * K
    for blk in range(3):
        t3[off + blk * Im: off + (blk + 1) * Im] = th[off + blk * Im: off + (blk + 1) * Im][comp]
    assert O.loglik(spec, y, t3)[0] == pytest.approx(base, rel=1e-12)


def test_test_functions_against_quadrature_and_simulator():
    tr = TRUTHS["k3i4"]
    spec = O.ModelSpec(K=3, I=4, gamma=True)
    th = I.theta_of_truth(tr)
    y, eps, h, v_T, h_next = I.simulate_egarch(tr, 200, seed=8, return_path=True)
    _, st = O.loglik(spec, y, th, with_state=True)
    g = O.testfn(spec, th, st)[0]
    # g1: log volatility at t = log h_t from the simulator
    assert g[0] == pytest.approx(math.log(h[-1]), rel=1e-10)
    # g2: E(eps^3) of the mixture by quadrature
    f = lambda e: e ** 3 * sum(p * stats.norm.pdf(e, m, s) for p, m, s in zip(tr.p, tr.mu, tr.sig))
    m3, _ = integrate.quad(f, -40, 40, limit=200)
    assert g[1] == pytest.approx(m3, abs=1e-9)
    # g3: P(Y_{t+1} < -0.03) with the simulator's h_{t+1} and scipy's normal cdf
    x = (-0.03 - tr.mu_y) / h_next
    p3 = sum(p * stats.norm.cdf(x, m, s) for p, m, s in zip(tr.p, tr.mu, tr.sig))
    assert g[2] == pytest.approx(p3, rel=1e-10)


def test_symmetric_mixture_has_zero_skewness():
    spec = O.ModelSpec(K=1, I=2, gamma=True)
    th = np.array([0.0, math.log(0.01), 1.0, -2.0, 0.0, 0.3, 0.3, 0.0, 0.0, -0.5, -0.5])
    g = O.testfn(spec, th, np.array([0.1, 0.2]))[0]
    assert abs(g[1]) < 1e-15


@pytest.mark.parametrize("name", ["k1i1", "k2i2", "k3i4"])
def test_gradient_matches_central_differences(name):
    tr = TRUTHS[name]
    spec = O.ModelSpec(K=tr.K, I=tr.I, gamma=True)
    rng = np.random.default_rng(4)
    th = I.theta_of_truth(tr) + rng.normal(0, 0.05, spec.d)
    y = I.simulate_egarch(tr, 150, seed=6)
    ll, g = O.loglik_grad(spec, y, th)
    assert ll[0] == pytest.approx(O.loglik(spec, y, th)[0], rel=1e-14)
    h = 1e-5
    fd = np.zeros(spec.d)
    for i in range(spec.d):
        e = np.zeros(spec.d)
        e[i] = h
        fd[i] = (O.loglik(spec, y, th + e)[0] - O.loglik(spec, y, th - e)[0]) / (2 * h)
    np.testing.assert_allclose(g[0], fd, rtol=2e-5, atol=2e-4)


def test_linreg_likelihood_and_gradient_closed_form():
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(80, beta, 0.7, seed=3)
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=0.7, prior_mean=np.zeros(3),
                       prior_sd=np.full(3, 2.0))
    b = np.array([0.4, -0.9, 2.1])
    want = stats.norm.logpdf(y, X @ b, 0.7).sum()
    assert O.loglik(spec, y, b, X=X)[0] == pytest.approx(want, rel=1e-13)
    _, g = O.loglik_grad(spec, y, b, X=X)
    np.testing.assert_allclose(g[0], X.T @ (y - X @ b) / 0.49, rtol=1e-11)


def test_range_continuation_equals_full_recursion():
    tr = TRUTHS["k2i2"]
    spec = O.ModelSpec(K=2, I=2, gamma=True)
    th = I.theta_of_truth(tr)
    y = I.simulate_egarch(tr, 120, seed=12)
    full, st_full = O.loglik(spec, y, th, with_state=True)
    a, st = O.loglik_range(spec, y, 0, 50, th, np.zeros(3))
    b, st = O.loglik_range(spec, y, 50, 120, th, st)
    assert a + b == pytest.approx(full[0], rel=1e-13)
    np.testing.assert_allclose(st, st_full[0], rtol=1e-13)
