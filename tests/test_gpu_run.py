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
    J, N = 32, 256
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
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    # log wtilde has no NSE of its own; its spread is that of log wbar
    assert abs(lt - lml) < 4 * nse
    mom = ctx.moments()
    for i in range(3):
        assert abs(mom[i, 0] - mn[i]) < 3 * mom[i, 2]
        assert mom[i, 1] == pytest.approx(math.sqrt(Vn[i, i]), rel=0.1)
    ctx.close()


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_linreg_independent_sampler_matches_closed_form(S, tempering):
    """Section 3.3's independent Gaussian sampler (proposal N(mean, V) of the
    population) reaches the exact log ML and posterior means; the hybrid
    design cannot be recorded for it."""
    X, y, m0, s0, lml, mn, Vn = _linreg()
    J, N = 32, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=J, N=N, precision=S.FP64, seed=12, mutation=S.INDEP,
                         tempering=S.POWER if tempering == "power" else S.DATA)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=6)
    ctx = S.init(m, c, y, th0, X=X)
    n, info = ctx.run()
    assert info["done"] == 1
    lm, nse, lt = ctx.log_ml()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    mom = ctx.moments()
    for i in range(3):
        assert abs(mom[i, 0] - mn[i]) < 3 * mom[i, 2]
    ctx.close()
    ctx = S.init(m, c, y, th0, X=X)
    with pytest.raises(S.SMCError):
        ctx.record_design()
    ctx.close()


def test_independent_sampler_egarch_matches_oracle_run(S):
    """FP64 EGARCH(1,1) run with the independent sampler: GPU and oracle agree
    on log ML within combined NSE."""
    w = I.WORKLOADS["egarch11_T500"]
    y = w.data()[:300]
    m = S.model_egarch(1, 1, False)
    mean, sd, lo = S.model_prior(m)
    J, N = 32, 128
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=71)
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, seed=3, mutation=S.INDEP), y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    ctx.close()
    spec = O.ModelSpec(K=1, I=1, gamma=False)
    r = O.smc_run(spec, y, th0, J, N, tempering=1, mutation=O.INDEP, seed=3, nthreads=8)
    assert r["status"] == 0
    comb = math.hypot(nse, r["log_ml_nse"])
    assert abs(lm - r["log_ml"]) < 3 * comb, (lm, r["log_ml"], comb)


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
    J, N = 32, 128
    m = S.model_egarch(1, 1, True, free_idx=[1], theta_fixed=th_true)
    c = S.config_default(J=J, N=N, precision=S.FP64 if precision == "fp64" else S.FP32, seed=3,
                         tempering=S.POWER if tempering == "power" else S.DATA)
    th0 = I.draw_prior([math.log(0.01)], [1.0], [-np.inf], J * N, seed=41)
    ctx = S.init(m, c, y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    mom = ctx.moments()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    assert abs(mom[0, 0] - pmean) < 3 * mom[0, 2]
    ctx.close()


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_egarch11_small_run_agrees_with_oracle(S, tempering):
    """EGARCH(1,1), Gaussian shocks, 4 parameters, T = 500, J = 4 x N = 256,
    FP64, 10 Metropolis steps per M phase: GPU and oracle runs agree on log ML
    and posterior means within 3 combined NSE.  With J = 4 a single run's NSE
    rests on 3 degrees of freedom, so each side runs 8 seeds (own prior draws
    and random numbers) and their averages are compared, with the NSE of an
    average sqrt(sum NSE_k^2) / 8."""
    w = I.WORKLOADS["egarch11_T500"]
    y = w.data()
    m = S.model_egarch(1, 1, False)
    mean, sd, lo = S.model_prior(m)
    spec = O.ModelSpec(K=1, I=1, gamma=False)
    tmode = S.POWER if tempering == "power" else S.DATA
    n = 8
    g_lm, g_n, o_lm, o_n = [], [], [], []
    g_m, g_mn, o_m, o_mn = [], [], [], []
    for k in range(n):
        th0 = I.draw_prior(mean, sd, lo, w.P, seed=w.prior_seed + 100 * k)
        c = S.config_default(J=w.J, N=w.N, precision=S.FP64, rbar=10, kappa=1, seed=7 + k, tempering=tmode)
        ctx = S.init(m, c, y, th0)
        ctx.run()
        lm, nse, _ = ctx.log_ml()
        mom = ctx.moments()
        ctx.close()
        g_lm.append(lm); g_n.append(nse); g_m.append(mom[:4, 0]); g_mn.append(mom[:4, 2])
        r = O.smc_run(spec, y, th0, w.J, w.N, rbar=10, kappa=1, seed=1007 + k, nthreads=8,
                      tempering=1 if tempering == "power" else 0)
        o_lm.append(r["log_ml"]); o_n.append(r["log_ml_nse"])
        mo = [O.moment(r["theta"][:, i], w.J, w.N) for i in range(4)]
        o_m.append([x[0] for x in mo]); o_mn.append([x[2] for x in mo])
    comb = math.sqrt(np.sum(np.square(g_n)) + np.sum(np.square(o_n))) / n
    assert abs(np.mean(g_lm) - np.mean(o_lm)) < 3 * comb, (np.mean(g_lm), np.mean(o_lm), comb)
    combm = np.sqrt(np.sum(np.square(g_mn), axis=0) + np.sum(np.square(o_mn), axis=0)) / n
    dm = np.abs(np.mean(g_m, axis=0) - np.mean(o_m, axis=0))
    assert np.all(dm < 3 * combm), (dm, combm)


def test_fp32_and_fp64_runs_agree(S):
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 1000, seed=8)
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 32, 256
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
    assert abs(l64 - l32) < 3 * math.hypot(n64, n32), (l64, l32, n64, n32)
    for f in range(m64.shape[0]):
        assert abs(m64[f, 0] - m32[f, 0]) < 3 * math.hypot(m64[f, 2], m32[f, 2]), f


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
    np.testing.assert_allclose(ll[pick], ll_o, rtol=1e-6)
    # the FP32 path evaluates the log prior in FP32 (FP32 mode reading)
    np.testing.assert_allclose(lp[pick], O.logprior(spec, th[pick]), rtol=1e-5)
    np.testing.assert_allclose(st[pick], st_o, rtol=2e-3, atol=2e-3)
    # the posterior concentrates near the data-generating parameters
    th_true = I.theta_of_truth(w.truth)
    assert abs(np.mean(th[:, 1]) - th_true[1]) < 0.2


def test_data_tempering_dates_of_interest(S):
    """A forced stop at a date of interest ends a cycle there even with RSS >= D1."""
    X, y, m0, s0, lml, mn, Vn = _linreg()
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=32, N=128, precision=S.FP64, tempering=S.DATA, seed=4, force_dates=[37, 45])
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 32 * 128, seed=6)
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
    assert abs(lm - lml) < 3 * nse
    ctx.close()


def test_rne_stopping_rule_run(S):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=32, N=128, precision=S.FP64, stop_rule=S.STOP_RNE, rmax=30, seed=4)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 32 * 128, seed=6)
    ctx = S.init(m, c, y, th0, X=X)
    infos = []
    while True:
        inf = ctx.cycle()
        if inf is None:
            break
        infos.append(inf)
    assert all(1 <= i["R"] <= 30 for i in infos)
    lm, nse, _ = ctx.log_ml()
    assert abs(lm - lml) < 3 * nse
    ctx.close()


@pytest.mark.parametrize("workload", ["egarch22_T5000", "egarch34_T20000"])
def test_launch_shapes_give_identical_runs(S, workload):
    """Every launch shape (blocks of any multiple of 32 threads up to 224, one
    or two particles per thread) computes each particle's proposal, recursion
    and decision exactly as one particle per thread in 128-thread blocks.  The
    K=3, I=4 case adds outlying observations, so that the mixture sums' tail
    fallback and rescaling run in both kernels."""
    w = I.WORKLOADS[workload]
    truth = w.truth
    y = I.simulate_egarch(truth, 700, seed=8)
    if w.I >= 3:
        y[::37] *= 12.0
    m = S.model_egarch(w.K, w.I, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 16, 300   # P = 4800: ragged against 64/128/256-particle tiles
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=9)
    out = []
    shapes = [(1, 128), (1, 64), (1, 32), (2, 32), (2, 64), (2, 128), (1, 96), (2, 224), (1, 224), (2, 160)]
    for ppt, thr in shapes:
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
    assert ppt in (1, 2) and thr % 32 == 0 and 32 <= thr <= 224 and ms > 0
    ctx.run()
    assert ctx.log_ml()[0] == pytest.approx(out[0][0][0], rel=1e-12, abs=1e-9)
    ctx.close()


@pytest.mark.parametrize("precision,record,tempering", [("fp32", False, "power"), ("fp64", True, "power"),
                                                        ("fp32", False, "data"), ("fp64", True, "data")])
def test_pipelined_run_equals_cycle_by_cycle(S, precision, record, tempering):
    """smc_run enqueues the next cycle's C phase (power tempering: with its S
    phase; data tempering: its first batch of chunks) behind each M phase, so
    one host round trip serves both; the same context stepped with smc_cycle
    synchronises after each phase.  Both must produce the same cycles,
    designs and particles bitwise, also when the run is split by
    max_cycles."""
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 600, seed=11)
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 8, 512
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=12)
    prec = S.FP32 if precision == "fp32" else S.FP64
    out = []
    tmp = S.POWER if tempering == "power" else S.DATA
    for mode in ("run", "split", "cycle"):
        ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, seed=7, tempering=tmp), y, th0)
        if record:
            ctx.record_design()
        infos = []
        if mode == "run":
            n, last = ctx.run()
            infos = [n, last["cycle"], last["phi"], last["t"], last["R"], last["h_tenths"], last["acc_rate"]]
        elif mode == "split":
            n1, _ = ctx.run(3)
            n2, last = ctx.run()
            infos = [n1 + n2, last["cycle"], last["phi"], last["t"], last["R"], last["h_tenths"], last["acc_rate"]]
        else:
            n, last = 0, None
            while True:
                info = ctx.cycle()
                if info is None:
                    break
                n, last = n + 1, info
                if info["done"]:
                    break
            infos = [n, last["cycle"], last["phi"], last["t"], last["R"], last["h_tenths"], last["acc_rate"]]
        design = ctx.design() if record else None
        out.append((infos, ctx.log_ml(), ctx.particles(), design))
        ctx.close()
    for infos, lml, parts, design in out[1:]:
        assert infos == out[0][0]
        assert lml == out[0][1]
        for a, b in zip(parts, out[0][2]):
            np.testing.assert_array_equal(a, b)
        if record:
            for k in ("x", "R", "L"):
                np.testing.assert_array_equal(design[k], out[0][3][k])


def test_small_blocks_fp64_and_invalid_shapes(S):
    """FP64 runs give the same particles with 32- and 96-thread blocks; shapes
    outside the supported set are rejected."""
    truth = I.WORKLOADS["egarch11_T500"].truth
    y = I.simulate_egarch(truth, 300, seed=2)
    m = S.model_egarch(1, 1, False)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, 4 * 100, seed=3)
    out = []
    for thr in (128, 32, 96):
        ctx = S.init(m, S.config_default(J=4, N=100, precision=S.FP64, seed=1), y, th0)
        ctx.set_launch_shape(1, thr)
        for _ in range(3):
            ctx.cycle()
        out.append(ctx.particles())
        if thr == 32:
            for bad in [(1, 100), (1, 256), (1, 0), (2, 32), (3, 64)]:   # FP64 has no paired shape
                with pytest.raises(S.SMCError):
                    ctx.set_launch_shape(*bad)
        ctx.close()
    for o in out[1:]:
        np.testing.assert_array_equal(out[0][0], o[0])
        np.testing.assert_array_equal(out[0][1], o[1])


# ---------------------------------------------- log score and PIT (Section 4.1)
def _prefix_lml(X, y, m0, s0, t):
    V0 = np.diag(s0 ** 2)
    return stats.multivariate_normal(X[:t] @ m0, np.eye(t) + X[:t] @ V0 @ X[:t].T).logpdf(y[:t])


def _predictive_cdf(X, y, m0, s0):
    Vinv, b = np.diag(1 / s0 ** 2), np.diag(1 / s0 ** 2) @ m0
    out = np.zeros(len(y))
    for s in range(len(y)):
        V = np.linalg.inv(Vinv)
        x = X[s]
        out[s] = stats.norm.cdf((y[s] - x @ (V @ b)) / math.sqrt(1.0 + x @ V @ x))
        Vinv = Vinv + np.outer(x, x)
        b = b + x * y[s]
    return out


def test_linreg_log_score_and_pit_match_closed_forms(S):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    b = 20
    J, N = 32, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    c = S.config_default(J=J, N=N, precision=S.FP64, seed=13, tempering=S.DATA, burnin=b, pit=1)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=7)
    ctx = S.init(m, c, y, th0, X=X)
    ts = []
    while True:
        info = ctx.cycle()
        ts.append(info["t"])
        if info["done"]:
            break
    assert b in ts
    ls, nse = ctx.log_score()
    exact = lml - _prefix_lml(X, y, m0, s0, b)
    assert abs(ls - exact) < 3 * nse, (ls, exact, nse)
    lm, lnse, _ = ctx.log_ml()
    assert abs(lm - lml) < 3 * lnse
    pit = ctx.pit()
    err = np.abs(pit - _predictive_cdf(X, y, m0, s0))
    assert np.all(np.isfinite(pit)) and err.max() < 0.08 and err.mean() < 0.02, (err.max(), err.mean())
    ctx.close()
    # the same prior draws give the oracle's PIT up to rounding through the first cycle
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=1.0, prior_mean=m0, prior_sd=s0)
    r = O.smc_run(spec, y, th0, J, N, X=X, tempering=0, pit=True, burnin=b, seed=13)
    t1 = ts[0]
    assert t1 == r["t"][0], (t1, r["t"][0])   # the first cycle stops where the oracle's does
    np.testing.assert_allclose(pit[:t1], r["pit"][:t1], rtol=0, atol=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_egarch_pit_first_cycle_matches_oracle(S, precision):
    """EGARCH(1,2): through the first cycle both sides weight the same prior
    draws, so the PIT values agree up to rounding (FP32: the indicator can flip
    only where the simulated and observed shocks tie to FP32 precision)."""
    tr = I.EgarchTruth(0.0, 0.01, (0.95,), (0.12,), (-0.05,))
    y = I.simulate_egarch(tr, 200, seed=41)
    m = S.model_egarch(1, 2, True)
    mean, sd, lo = S.model_prior(m)
    J, N = 8, 512
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=42)
    prec = S.FP64 if precision == "fp64" else S.FP32
    ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, seed=9, tempering=S.DATA, pit=1), y, th0)
    tg = ctx.cycle()["t"]
    pit = ctx.pit()
    ctx.close()
    assert np.all(np.isfinite(pit[:tg])) and np.all(np.isnan(pit[tg:]))   # not yet reached
    spec = O.ModelSpec(K=1, I=2, gamma=True)
    r = O.smc_run(spec, y, th0, J, N, tempering=0, pit=True, seed=9, max_cycles=1)
    t1 = tg
    assert t1 == r["t"][0], (t1, r["t"][0])   # the first cycle stops where the oracle's does
    tol = 1e-9 if precision == "fp64" else 2e-3
    np.testing.assert_allclose(pit[:t1], r["pit"][:t1], rtol=0, atol=tol)


def test_log_score_and_pit_need_data_tempering(S):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    m = S.model_linreg(3, 1.0, m0, s0)
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 2 * 64, seed=7)
    for kw in (dict(burnin=10), dict(pit=1)):
        with pytest.raises(S.SMCError):
            S.init(m, S.config_default(J=2, N=64, precision=S.FP64, tempering=S.POWER, **kw), y, th0, X=X)
    with pytest.raises(S.SMCError):
        S.init(m, S.config_default(J=2, N=64, precision=S.FP64, tempering=S.DATA, burnin=len(y)), y, th0, X=X)
    ctx = S.init(m, S.config_default(J=2, N=64, precision=S.FP64, tempering=S.DATA), y, th0, X=X)
    with pytest.raises(S.SMCError):
        ctx.pit()
    with pytest.raises(S.SMCError):
        ctx.log_score()
    ctx.close()


def test_nse_coverage_over_seeds_on_gpu(S):
    """Proposition 1: over 200 independent seeds the GPU runs' posterior-mean
    and log-ML errors, standardized by their NSE, cover the closed forms at
    about the t(J-1) rate (two-sided 95%, binomial tolerance)."""
    X, y, m0, s0, lml, mn, Vn = _linreg(T=40, seed=8)
    J, N = 8, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    tq = stats.t(J - 1).ppf(0.975)
    hits_m = hits_ml = 0
    n = 200
    for s in range(n):
        th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=3000 + s)
        ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, seed=700 + s, rbar=10), y, th0, X=X)
        ctx.run()
        lm, nse, _ = ctx.log_ml()
        mom = ctx.moments()
        ctx.close()
        hits_m += abs(mom[0, 0] - mn[0]) < tq * mom[0, 2]
        hits_ml += abs(lm - lml) < tq * nse
    # binomial(200, 0.95): mean 190, sd 3.1
    assert hits_m >= 175, hits_m
    assert hits_ml >= 160, hits_ml   # the log-ML normal approximation is the weaker one (ML_se)


# ----------------------------------------------------------- checkpoint/resume
@pytest.mark.parametrize("case", ["egarch_fp32_power", "linreg_data_score_pit", "egarch_mala", "hybrid_replay"])
def test_checkpoint_resume_continues_the_run_exactly(S, tmp_path, case):
    """A run saved between cycles and resumed in a new context ends with
    bitwise the same particles, log ML and auxiliary outputs as the run that
    went on uninterrupted (counter-based random numbers)."""
    if case == "linreg_data_score_pit":
        X, y, m0, s0, lml, mn, Vn = _linreg()
        m = S.model_linreg(3, 1.0, m0, s0)
        c = S.config_default(J=8, N=256, precision=S.FP64, seed=21, tempering=S.DATA, burnin=20, pit=1)
        th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), 8 * 256, seed=22)
        make = lambda: S.init(m, c, y, th0, X=X)
    else:
        tr = I.EgarchTruth(0.0, 0.01, (0.95,), (0.12,), (-0.05,))
        y = I.simulate_egarch(tr, 400, seed=23)
        m = S.model_egarch(1, 2, True)
        mean, sd, lo = S.model_prior(m)
        th0 = I.draw_prior(mean, sd, lo, 8 * 256, seed=24)
        mut = S.MALA if case == "egarch_mala" else S.RW
        c = S.config_default(J=8, N=256, precision=S.FP32, seed=25, mutation=mut,
                             acc_target=0.5 if mut == S.MALA else 0.25)
        make = lambda: S.init(m, c, y, th0)
    design = None
    if case == "hybrid_replay":
        ctx = make()
        ctx.record_design()
        ctx.run()
        design = ctx.design()
        ctx.close()

    def fresh():
        ctx = make()
        if design is not None:
            ctx.replay_design(design)
        return ctx

    path = tmp_path / "run.ckpt"
    a = fresh()
    for _ in range(3):
        a.cycle()
    a.save(path)
    a.run()
    b = S.load(path)
    b.run()
    for u, v in zip(a.particles(), b.particles()):
        assert np.array_equal(u, v)
    assert a.log_ml() == b.log_ml()
    if case == "linreg_data_score_pit":
        assert a.log_score() == b.log_score()
        assert np.array_equal(a.pit(), b.pit())
    a.close()
    b.close()


def test_run_from_device_prior_draws_matches_closed_form(S):
    """A run started from device prior draws (smc_draw_prior, theta0 on the
    device) reaches the regression's exact log ML."""
    X, y, m0, s0, lml, mn, Vn = _linreg()
    J, N = 32, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    th0 = S.draw_prior(m, 17, J * N)
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, seed=18), y, th0, X=X, theta0_on_device=True)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    ctx.close()
