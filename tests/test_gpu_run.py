"""Full simulator runs on the GPU through the C ABI, checked against closed
forms (conjugate regression, one-parameter quadrature) and against the oracle
run on the same workload, within combined numerical standard errors; plus
sampled parity of the final particles at the full benchmark size."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_1304_4334_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch_cuda()
    from paper_1304_4334_gb300 import build
    build.build()
    from paper_1304_4334_gb300 import smc
    return smc


def _linreg(T=60, seed=3):
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(T, beta, 1.0, seed=seed)
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    V0 = np.diag(s0 ** 2)
    lml = stats.multivariate_normal(X @ m0, np.eye(T) + X @ V0 @ X.T).logpdf(y)
    Vn = np.linalg.inv(np.linalg.inv(V0) + X.T @ X)
    mn = Vn @ (X.T @ y)
    return X, y, m0, s0, lml, mn, Vn


@pytest.mark.parametrize("resampler,tempering", [("residual", "power"), ("multinomial", "power"),
                                                ("residual", "data"), ("stratified", "power"),
                                                ("systematic", "data")])
def test_linreg_run_matches_closed_form(S, resampler, tempering):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    J, N = 16, 512
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=J, N=N, precision=S.FP64, seed=11,
                         tempering=S.POWER if tempering == "power" else S.DATA,
                         resampler={"residual": S.RESIDUAL, "multinomial": S.MULTINOMIAL,
                                    "stratified": S.STRATIFIED, "systematic": S.SYSTEMATIC}[resampler])
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=5)
    ctx = S.init(m, c, y, th0, X=X)
    n, info = ctx.run()
    assert info["done"] == 1 and info["phi"] == 1.0
    if tempering == "data":
        assert info["t"] == len(y)
    lm, nse, lt = ctx.log_ml()
    assert abs(lm - lml) < 3.5 * nse + 0.02, (lm, lml, nse)
    assert abs(lt - lml) < 5 * nse + 0.03
    mom = ctx.moments()
    for i in range(3):
        assert abs(mom[i, 0] - mn[i]) < 3.5 * mom[i, 2] + 1e-4
        assert mom[i, 1] == pytest.approx(math.sqrt(Vn[i, i]), rel=0.1)
    ctx.close()


@pytest.mark.parametrize("precision,tempering", [("fp64", "power"), ("fp32", "power"), ("fp32", "data")])
def test_one_parameter_egarch_matches_quadrature(S, precision, tempering):
    tr = I.EgarchTruth(0.0, 0.01, (0.95,), (0.12,), (-0.05,))
    y = I.simulate_egarch(tr, 300, seed=31)
    th_true = I.theta_of_truth(tr)
    spec = O.ModelSpec(K=1, I=1, gamma=True, free_idx=[1], theta_fixed=th_true)
    grid = np.linspace(math.log(0.01) - 2.0, math.log(0.01) + 2.0, 40001)
    lj = O.loglik(spec, y, grid[:, None], nthreads=4) + O.logprior(spec, grid[:, None])
    mx = lj.max()
    wq = np.exp(lj - mx)
    dx = grid[1] - grid[0]
    Z = integrate.simpson(wq, dx=dx)
    lml = mx + math.log(Z)
    pmean = integrate.simpson(wq * grid, dx=dx) / Z
    J, N = 16, 256
    m = S.model_egarch(1, 1, True, free_idx=[1], theta_fixed=th_true)
    c = S.config_default(J=J, N=N, precision=S.FP64 if precision == "fp64" else S.FP32, seed=3,
                         tempering=S.POWER if tempering == "power" else S.DATA)
    th0 = I.draw_prior([math.log(0.01)], [1.0], [-np.inf], J * N, seed=41)
    ctx = S.init(m, c, y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    mom = ctx.moments()
    assert abs(lm - lml) < 3.5 * nse + 0.01, (lm, lml, nse)
    assert abs(mom[0, 0] - pmean) < 3.5 * mom[0, 2] + 1e-4
    ctx.close()


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_egarch11_small_run_agrees_with_oracle(S, tempering):
    """EGARCH(1,1), Gaussian shocks, 4 parameters, T = 500, J = 4 x N = 256,
    FP64, 10 Metropolis steps per M phase: GPU and oracle runs agree on log ML
    and posterior means within combined NSE."""
    w = I.WORKLOADS["egarch11_T500"]
    y = w.data()
    m = S.model_egarch(1, 1, False)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed)
    tmode = S.POWER if tempering == "power" else S.DATA
    c = S.config_default(J=w.J, N=w.N, precision=S.FP64, rbar=10, kappa=1, seed=7, tempering=tmode)
    ctx = S.init(m, c, y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    mom = ctx.moments()
    ctx.close()
    spec = O.ModelSpec(K=1, I=1, gamma=False)
    r = O.smc_run(spec, y, th0, w.J, w.N, rbar=10, kappa=1, seed=7, nthreads=8,
                  tempering=1 if tempering == "power" else 0)
    tol = lambda a, b: 4.0 * math.hypot(a, b) + 0.02
    assert abs(lm - r["log_ml"]) < tol(nse, r["log_ml_nse"]), (lm, r["log_ml"], nse, r["log_ml_nse"])
    for i in range(4):
        mo, _, no, _ = O.moment(r["theta"][:, i], w.J, w.N)
        assert abs(mom[i, 0] - mo) < tol(mom[i, 2], no) + 1e-3, (i, mom[i], mo, no)


def test_fp32_and_fp64_runs_agree(S):
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 1000, seed=8)
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 16, 512
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=9)
    res = {}
    for prec in (S.FP64, S.FP32):
        c = S.config_default(J=J, N=N, precision=prec, seed=13 + prec)
        ctx = S.init(m, c, y, th0)
        ctx.run()
        res[prec] = (ctx.log_ml(), ctx.moments())
        ctx.close()
    (l64, n64, _), m64 = res[S.FP64]
    (l32, n32, _), m32 = res[S.FP32]
    assert abs(l64 - l32) < 4 * math.hypot(n64, n32) + 0.05, (l64, l32, n64, n32)
    for f in range(m64.shape[0]):
        assert abs(m64[f, 0] - m32[f, 0]) < 4 * math.hypot(m64[f, 2], m32[f, 2]) + 1e-3, f


def test_full_size_run_sampled_parity(S):
    """The benchmark workload (K=2, I=2, T=5000, J=64 x N=1024, FP32) run to
    the posterior; the final particles' log likelihood and log prior are
    recomputed one by one by the oracle for a sample of particles."""
    w = I.WORKLOADS["egarch22_T5000"]
    y = w.data()
    m = S.model_egarch(w.K, w.I, w.gamma)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed)
    c = S.config_default(J=w.J, N=w.N, precision=S.FP32, seed=1)
    ctx = S.init(m, c, y, th0)
    n, info = ctx.run()
    assert info["done"] == 1 and 5 < n < 400
    lm, nse, lt = ctx.log_ml()
    assert math.isfinite(lm) and 0 < nse < 5 and abs(lt - lm) < 10 * nse + 1
    th, ll, lp, st = ctx.particles()
    ctx.close()
    spec = O.ModelSpec(K=w.K, I=w.I, gamma=w.gamma)
    pick = np.random.default_rng(0).choice(w.P, 48, replace=False)
    ll_o, st_o = O.loglik(spec, y, th[pick], with_state=True, nthreads=8)
    np.testing.assert_allclose(ll[pick], ll_o, rtol=1e-4)
    np.testing.assert_allclose(lp[pick], O.logprior(spec, th[pick]), rtol=1e-12)
    np.testing.assert_allclose(st[pick], st_o, rtol=2e-3, atol=2e-3)
    # the posterior concentrates near the data-generating parameters
    th_true = I.theta_of_truth(w.truth)
    assert abs(np.mean(th[:, 1]) - th_true[1]) < 0.2


def test_data_tempering_dates_of_interest(S):
    """A forced stop at a date of interest ends a cycle there even with RSS >= D1."""
    X, y, m0, s0, lml, mn, Vn = _linreg()
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=8, N=256, precision=S.FP64, tempering=S.DATA, seed=4, force_dates=[37, 45])
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 8 * 256, seed=6)
    ctx = S.init(m, c, y, th0, X=X)
    ts = []
    while True:
        inf = ctx.cycle()
        if inf is None:
            break
        ts.append(inf["t"])
    assert 37 in ts and 45 in ts and ts[-1] == len(y)
    assert all(b > a for a, b in zip(ts, ts[1:]))
    lm, nse, _ = ctx.log_ml()
    assert abs(lm - lml) < 4 * nse + 0.02
    ctx.close()


def test_rne_stopping_rule_run(S):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=8, N=256, precision=S.FP64, stop_rule=S.STOP_RNE, rmax=30, seed=4)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 8 * 256, seed=6)
    ctx = S.init(m, c, y, th0, X=X)
    infos = []
    while True:
        inf = ctx.cycle()
        if inf is None:
            break
        infos.append(inf)
    assert all(1 <= i["R"] <= 30 for i in infos)
    lm, nse, _ = ctx.log_ml()
    assert abs(lm - lml) < 4 * nse + 0.02
    ctx.close()


def test_launch_shapes_give_identical_runs(S):
    """Two particles per thread (either block size) computes every particle's
    proposal, recursion and decision exactly as one particle per thread."""
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 700, seed=8)
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 16, 300   # P = 4800: ragged against 64/128/256-particle tiles
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=9)
    out = []
    for ppt, thr in [(1, 128), (2, 64), (2, 128)]:
        ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP32, seed=5), y, th0)
        ctx.set_launch_shape(ppt, thr)
        ctx.run()
        out.append((ctx.log_ml(), ctx.particles()))
        ctx.close()
    for (lm, (th, ll, lp, st)) in out[1:]:
        assert lm[0] == pytest.approx(out[0][0][0], rel=1e-12, abs=1e-9)
        np.testing.assert_allclose(th, out[0][1][0], rtol=0, atol=1e-10)
        np.testing.assert_allclose(ll, out[0][1][1], rtol=1e-12)
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP32, seed=5), y, th0)
    ppt, thr, ms = ctx.autotune(iters=1)
    assert (ppt, thr) in [(1, 128), (2, 64), (2, 128)] and ms > 0
    ctx.run()
    assert ctx.log_ml()[0] == pytest.approx(out[0][0][0], rel=1e-12, abs=1e-9)
    ctx.close()
