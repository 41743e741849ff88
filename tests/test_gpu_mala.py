"""GPU parity of the adjoint gradient kernel and the MALA mutation (through the
C ABI) against the oracle's forward-mode gradient and MALA step, central finite
differences in FP64 (h = 1e-5), the autograd wrapper, and full MALA runs
against closed forms."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

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


def _grad_case(S, K, I_, gamma, T, P, precision, seed):
    torch = torch_cuda()
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=seed)
    spec = O.ModelSpec(K=K, I=I_, gamma=gamma)
    th = particles(spec.d, truth, K, I_, gamma, P, seed + 3)
    ll_o, g_o = O.loglik_grad(spec, y, th)
    m = S.model_egarch(K, I_, gamma)
    obs = dev(y, torch.float32 if precision == S.FP32 else torch.float64)
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    g = torch.empty((spec.d, P), dtype=torch.float64, device="cuda")
    S.loglik_grad(m, precision, obs, soa(th), ll, g)
    torch.cuda.synchronize()
    return spec, y, th, ll_o, g_o, host(ll), host(g).T


@pytest.mark.parametrize("K,I_,gamma", SHAPES)
@pytest.mark.parametrize("T,P", [(1, 7), (33, 129), (517, 200)])
def test_gradient_fp64_matches_oracle(S, K, I_, gamma, T, P):
    spec, y, th, ll_o, g_o, ll, g = _grad_case(S, K, I_, gamma, T, P, S.FP64, seed=11 + T)
    np.testing.assert_allclose(ll, ll_o, rtol=1e-9)
    scale = np.abs(g_o).max(axis=1, keepdims=True) + 1.0
    np.testing.assert_allclose(g, g_o, rtol=1e-7, atol=1e-9 * scale.max())


@pytest.mark.parametrize("K,I_,gamma", [(1, 1, True), (2, 2, True), (3, 4, True)])
def test_gradient_fp32_matches_oracle(S, K, I_, gamma):
    spec, y, th, ll_o, g_o, ll, g = _grad_case(S, K, I_, gamma, 1200, 300, S.FP32, seed=7)
    np.testing.assert_allclose(ll, ll_o, rtol=1e-4)
    # FP32 recursion and per-segment FP32 sums: 2e-3 of each particle's largest component
    scale = np.abs(g_o).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - g_o) <= 2e-3 * scale + 1e-3), (np.abs(g - g_o) / scale).max()


def test_gradient_fp64_matches_central_differences(S):
    """Central differences of the GPU FP64 likelihood kernel at h = 1e-5."""
    torch = torch_cuda()
    K, I_, T, P = 2, 2, 800, 16
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=3)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 5)
    m = S.model_egarch(K, I_, True)
    obs = dev(y)
    ll = torch.empty(P, dtype=torch.float64, device="cuda")
    g = torch.empty((spec.d, P), dtype=torch.float64, device="cuda")
    S.loglik_grad(m, S.FP64, obs, soa(th), ll, g)
    g = host(g).T
    h = 1e-5
    fd = np.zeros_like(g)
    for i in range(spec.d):
        e = np.zeros(spec.d)
        e[i] = h
        lp_ = torch.empty(P, dtype=torch.float64, device="cuda")
        lm_ = torch.empty(P, dtype=torch.float64, device="cuda")
        S.loglik(m, S.FP64, obs, soa(th + e), lp_)
        S.loglik(m, S.FP64, obs, soa(th - e), lm_)
        fd[:, i] = (host(lp_) - host(lm_)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=2e-4)


def test_gradient_fixed_parameters_and_linreg(S):
    torch = torch_cuda()
    truth = egarch_truth(2, 2)
    y = I.simulate_egarch(truth, 400, seed=9)
    th_true = I.theta_of_truth(truth)
    free = [1, 3, 9, 12]
    spec = O.ModelSpec(K=2, I=2, gamma=True, free_idx=free, theta_fixed=th_true)
    m = S.model_egarch(2, 2, True, free_idx=free, theta_fixed=th_true)
    th = th_true[free] + 0.03 * np.random.default_rng(1).standard_normal((50, 4))
    ll_o, g_o = O.loglik_grad(spec, y, th)
    ll = torch.empty(50, dtype=torch.float64, device="cuda")
    g = torch.empty((4, 50), dtype=torch.float64, device="cuda")
    S.loglik_grad(m, S.FP64, dev(y), soa(th), ll, g)
    np.testing.assert_allclose(host(ll), ll_o, rtol=1e-9)
    np.testing.assert_allclose(host(g).T, g_o, rtol=1e-7, atol=1e-7)
    beta = np.array([0.5, -1.0, 2.0])
    X, yr = I.linreg_data(150, beta, 0.8, seed=2)
    specl = O.ModelSpec(model=O.LINREG, p=3, sigma=0.8, prior_mean=np.zeros(3), prior_sd=np.full(3, 2.0))
    ml = S.model_linreg(3, 0.8, np.zeros(3), np.full(3, 2.0))
    rec = np.zeros((150, S.linreg_width(3)))
    rec[:, :3] = X
    rec[:, 3] = yr
    thl = beta + 0.1 * np.random.default_rng(2).standard_normal((64, 3))
    ll = torch.empty(64, dtype=torch.float64, device="cuda")
    g = torch.empty((3, 64), dtype=torch.float64, device="cuda")
    S.loglik_grad(ml, S.FP64, dev(rec), soa(thl), ll, g)
    lo, go = O.loglik_grad(specl, yr, thl, X=X)
    np.testing.assert_allclose(host(ll), lo, rtol=1e-12)
    np.testing.assert_allclose(host(g).T, go, rtol=1e-10, atol=1e-10)


def test_autograd_function(S):
    torch = torch_cuda()
    from paper_1304_4334_gb300.autograd import loglik
    K, I_, T, P = 2, 2, 300, 40
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=4)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 6)
    m = S.model_egarch(K, I_, True)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.linspace(0.5, 1.5, P, dtype=torch.float64, device="cuda")
    out = (loglik(theta, m, S.FP64, dev(y)) * w).sum()
    out.backward()
    ll_o, g_o = O.loglik_grad(spec, y, th)
    assert out.item() == pytest.approx(float((ll_o * host(w)).sum()), rel=1e-10)
    np.testing.assert_allclose(host(theta.grad), g_o * host(w)[:, None], rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mala_step_matches_oracle(S, precision):
    torch = torch_cuda()
    prec = S.FP64 if precision == "fp64" else S.FP32
    K, I_, T, P = 2, 2, 300, 777
    truth = egarch_truth(K, I_)
    y = I.simulate_egarch(truth, T, seed=21)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    th = particles(spec.d, truth, K, I_, True, P, 23)
    ll, g = O.loglik_grad(spec, y, th)
    _, st = O.loglik(spec, y, th, with_state=True)
    lp = O.logprior(spec, th)
    _, V = O.mean_cov(th)
    Lm, _ = O.cholesky(0.8 ** 2 * V)
    phi, seed, cycle, it = 0.8, 31, 2, 5
    th_o, ll_o, lp_o, g_o, st_o, acc_o, n_o = O.mutate_mala(spec, y, th, ll, lp, g, st, Lm, phi, seed,
                                                            cycle, it, nthreads=8)
    m = S.model_egarch(K, I_, True)
    obs = dev(y, torch.float32 if prec == S.FP32 else torch.float64)
    tg, llg, lpg, gg, stg = soa(th), dev(ll), dev(lp), soa(g), soa(st)
    n = S.mutate_mala(m, prec, obs, tg, llg, lpg, gg, stg, dev(Lm), phi, seed, cycle, it)
    th_g = host(tg).T
    acc_g = np.any(th_g != th, axis=1)
    assert n == acc_g.sum()
    diff = acc_g != acc_o.astype(bool)
    limit = 2 if prec == S.FP64 else max(3, P // 50)
    assert diff.sum() <= limit, diff.sum()
    same = ~diff
    tol = 1e-9 if prec == S.FP64 else 1e-4
    np.testing.assert_allclose(th_g[same], th_o[same], rtol=tol, atol=1e-12 if prec == S.FP64 else 1e-5)
    np.testing.assert_allclose(host(llg)[same], ll_o[same], rtol=tol)
    gsc = np.abs(g_o[same]).max(axis=1, keepdims=True)
    assert np.all(np.abs(host(gg).T[same] - g_o[same]) <= (1e-7 if prec == S.FP64 else 2e-3) * gsc + 1e-6)
    assert 0.05 < n / P <= 1.0


def _linreg():
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(60, beta, 1.0, seed=3)
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    V0 = np.diag(s0 ** 2)
    lml = stats.multivariate_normal(X @ m0, np.eye(60) + X @ V0 @ X.T).logpdf(y)
    Vn = np.linalg.inv(np.linalg.inv(V0) + X.T @ X)
    mn = Vn @ (X.T @ y)
    return X, y, m0, s0, lml, mn, Vn


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_mala_linreg_run_matches_closed_form(S, tempering):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    J, N = 32, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=J, N=N, precision=S.FP64, mutation=S.MALA, acc_target=0.5, seed=17,
                         tempering=S.POWER if tempering == "power" else S.DATA)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=5)
    ctx = S.init(m, c, y, th0, X=X)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    mom = ctx.moments()
    ctx.close()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    for i in range(3):
        assert abs(mom[i, 0] - mn[i]) < 3 * mom[i, 2]
        assert mom[i, 1] == pytest.approx(math.sqrt(Vn[i, i]), rel=0.1)


def test_mala_one_parameter_egarch_matches_quadrature(S):
    tr = I.EgarchTruth(0.0, 0.01, (0.95,), (0.12,), (-0.05,))
    y = I.simulate_egarch(tr, 300, seed=31)
    th_true = I.theta_of_truth(tr)
    spec = O.ModelSpec(K=1, I=1, gamma=True, free_idx=[1], theta_fixed=th_true)
    grid = np.linspace(math.log(0.01) - 2.0, math.log(0.01) + 2.0, 40001)
    lj = O.loglik(spec, y, grid[:, None], nthreads=4) + O.logprior(spec, grid[:, None])
    mx = lj.max()
    wq = np.exp(lj - mx)
    Z = integrate.simpson(wq, dx=grid[1] - grid[0])
    lml = mx + math.log(Z)
    pmean = integrate.simpson(wq * grid, dx=grid[1] - grid[0]) / Z
    J, N = 32, 128
    m = S.model_egarch(1, 1, True, free_idx=[1], theta_fixed=th_true)
    c = S.config_default(J=J, N=N, precision=S.FP32, mutation=S.MALA, acc_target=0.5, seed=3)
    th0 = I.draw_prior([math.log(0.01)], [1.0], [-np.inf], J * N, seed=41)
    ctx = S.init(m, c, y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    mom = ctx.moments()
    ctx.close()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    assert abs(mom[0, 0] - pmean) < 3 * mom[0, 2]


def test_mala_and_rw_runs_agree(S):
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 800, seed=8)
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 32, 256
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=9)
    res = {}
    for mut in (S.RW, S.MALA):
        c = S.config_default(J=J, N=N, precision=S.FP32, seed=21 + mut, mutation=mut,
                             acc_target=0.25 if mut == S.RW else 0.5)
        ctx = S.init(m, c, y, th0)
        ctx.run()
        res[mut] = (ctx.log_ml(), ctx.moments())
        ctx.close()
    (lr, nr, _), mr = res[S.RW]
    (lm_, nm, _), mm = res[S.MALA]
    assert abs(lr - lm_) < 3 * math.hypot(nr, nm), (lr, lm_, nr, nm)
    for f in range(mr.shape[0]):
        assert abs(mr[f, 0] - mm[f, 0]) < 3 * math.hypot(mr[f, 2], mm[f, 2]), f
