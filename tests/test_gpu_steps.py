"""Steps of the simulator that a whole run cannot see, checked on the GPU
against the oracle through the C ABI.

A wrong proposal covariance, step size, iteration count or C-phase stopping
point leaves the posterior invariant, so the closed-form run tests stay green
with any of them.  Each is compared here with what the paper's rule gives for
the same particles:

- the first cycle from identical prior draws (Algorithm 1 step 2(a); Section
  3.3 "C phase termination"; Section 4.2): the data-tempering stop t_1, the
  power-tempering increment, the pooled RSS and every group's log wbar_j(0);
- the proposal covariance inside a run (Section 3.3 "Metropolis steps",
  Sigma = h^2 V): the Cholesky factor the run recorded for an iteration
  against the oracle's factor of h^2 times the pooled covariance of the
  particles entering that iteration (first iteration of an M phase: sums formed
  by the S-phase gather; later iterations: by the previous mutation launch);
- the step-size rule (h up or down one tenth on the pooled acceptance rate
  against the target, clamped to [0.1, 1]) and both stopping rules (Section 3.3
  "M phase Termination").

The particles entering iteration r of cycle l come from a replay of the run's
own recorded design (Algorithm 3) with the same seed, cut after r iterations
of cycle l.  A same-seed replay reproduces the adaptive run bit for bit
(test_gpu_hybrid.py), so the cut replay holds exactly the particles the
adaptive run had at that point; the expected factor, step size and stopping
decision are then computed from them by the oracle.
"""

import numpy as np
import pytest

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


# --------------------------------------------------------------- helpers
def _cut(design, ell, r):
    """The design of cycles 1..ell with cycle ell stopped after r iterations."""
    R = np.array(design["R"][:ell], dtype=np.int32)
    R[ell - 1] = r
    return {"x": np.array(design["x"][:ell]), "R": R, "L": design["L"][:int(R.sum())]}


def _snapshot(ctx, th0, seed, design, ell, r):
    """Particles of the adaptive run entering iteration r of cycle ell (r = R_ell:
    at the end of the cycle)."""
    ctx.reset(th0, seed)
    ctx.replay_design(_cut(design, ell, r))
    for _ in range(ell):
        assert ctx.cycle() is not None
    return ctx.particles()


def _adaptive(S, m, cfg, y, th0):
    ctx = S.init(m, cfg, y, th0)
    ctx.record_design(8192)
    infos = []
    while True:
        info = ctx.cycle()
        if info is None:
            break
        infos.append(info)
    design = ctx.design()
    ctx.close()
    assert sum(i["R"] for i in infos) == design["L"].shape[0]
    return infos, design


def _row_scaled_err(Lg, Lo):
    """max_ij |Lg - Lo|_ij / ||row i of Lo||: the error of each entry against the
    scale of its row (the standard deviation of that proposal component)."""
    rn = np.sqrt((Lo ** 2).sum(axis=1))
    return float((np.abs(np.tril(Lg) - np.tril(Lo)) / rn[:, None]).max())


def _h_tenths_of(Lg, V):
    """The step size (in tenths) that makes Lg = h chol(V): Sigma = h^2 V."""
    Lv, z = O.cholesky(V)
    assert z == 0
    ratio = np.diag(Lg) / np.diag(Lv)
    k = int(round(10.0 * float(np.median(ratio))))
    return k, Lv


# ------------------------------------------------- first cycle (C phase, a_j)
def _rss(logw):
    m = logw.max()
    w = np.exp(logw - m)
    return w.sum() ** 2 / (len(w) * (w * w).sum())


def _group_logmean(logw, J, N):
    lw = logw.reshape(J, N)
    m = lw.max(axis=1, keepdims=True)
    return (m[:, 0] + np.log(np.exp(lw - m).mean(axis=1)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_first_cycle_data_tempering_matches_oracle(S, precision):
    """Data tempering from identical prior draws: the GPU stops the first C phase
    at the oracle's t_1 (the first t with RSS < D1), with the pooled RSS and each
    group's log wbar_j(0) = log N^-1 sum_n exp(sum_{s<=t_1} l_s(theta_jn)) of the
    definition (Algorithm 1 step 2(a); Section 4.2), and a_j = log wbar_j(0)."""
    K, I_ = 2, 2
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 600, seed=8)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    J, N = 16, 256
    th0 = O.draw_prior(spec, 77, J * N)
    # oracle: per-observation terms, cumulative log weights, RSS path
    terms = np.stack([O.loglik_terms(spec, y, th0[n]) for n in range(J * N)])
    cum = np.cumsum(np.where(np.isfinite(terms), terms, -np.inf), axis=1)
    rss = np.array([_rss(cum[:, t]) for t in range(60)])
    t1 = int(np.argmax(rss < 0.5)) + 1
    assert rss[t1 - 1] < 0.5 and (t1 == 1 or rss[t1 - 2] >= 0.5)
    # the stopping point is unambiguous at FP32 precision of the weights
    assert abs(rss[t1 - 1] - 0.5) > 1e-3 and (t1 == 1 or abs(rss[t1 - 2] - 0.5) > 1e-3)
    r = O.smc_run(spec, y, th0, J, N, tempering=0, max_cycles=1, seed=5, nthreads=8)
    assert r["t"][0] == t1
    m = S.model_egarch(K, I_, True)
    prec = S.FP64 if precision == "fp64" else S.FP32
    ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, tempering=S.DATA, seed=5), y, th0)
    info = ctx.cycle()
    a, lw = ctx.group_estimators()
    ctx.close()
    assert info["t"] == t1, (info["t"], t1)
    ref_lw = _group_logmean(cum[:, t1 - 1], J, N)
    tol = 1e-9 if precision == "fp64" else 2e-4
    # the data-tempering stop statistic weighs with FP32 exponentials of FP64
    # log-weight differences (~1e-7 relative)
    rtol = 1e-6 if precision == "fp64" else 2e-4
    assert info["rss"] == pytest.approx(rss[t1 - 1], rel=rtol)
    assert info["rss"] == pytest.approx(r["rss"][0], rel=rtol)
    np.testing.assert_allclose(lw, ref_lw, rtol=tol, atol=tol)
    np.testing.assert_allclose(a, lw, rtol=0, atol=0)
    np.testing.assert_allclose(a, r["a"], rtol=tol, atol=tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_first_cycle_power_tempering_matches_oracle(S, precision):
    """Power tempering from identical prior draws: the increment solves
    RSS(dphi) = D1 (the oracle's bisection), and at the GPU's increment the
    pooled RSS and each group's log wbar_j(0) = log N^-1 sum_n exp(dphi l_n) equal
    the definition evaluated on the oracle's FP64 log likelihoods."""
    K, I_ = 2, 2
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 2000, seed=8)
    spec = O.ModelSpec(K=K, I=I_, gamma=True)
    J, N = 32, 512
    th0 = O.draw_prior(spec, 78, J * N)
    ll = O.loglik(spec, y, th0, nthreads=8)
    dphi_o, rss_o = O.power_search(ll, 0.0)
    m = S.model_egarch(K, I_, True)
    prec = S.FP64 if precision == "fp64" else S.FP32
    ctx = S.init(m, S.config_default(J=J, N=N, precision=prec, tempering=S.POWER, seed=5), y, th0)
    info = ctx.cycle()
    a, lw = ctx.group_estimators()
    ctx.close()
    dphi = info["phi"]
    assert dphi == pytest.approx(dphi_o, rel=1e-5), (dphi, dphi_o)
    lwn = np.where(np.isfinite(ll), dphi * ll, -np.inf)
    # the GPU's FP32 log likelihoods of raw prior draws carry ~1e-4 relative error
    tol = 1e-9 if precision == "fp64" else 1e-3
    assert info["rss"] == pytest.approx(_rss(lwn), rel=tol)
    assert abs(info["rss"] - 0.5) < 1e-5
    np.testing.assert_allclose(lw, _group_logmean(lwn, J, N), rtol=tol, atol=tol)
    np.testing.assert_allclose(a, lw, rtol=0, atol=0)


# ---------------------------------------- in-run covariance and the h rule
@pytest.mark.parametrize("shape", ["egarch22_T5000", "egarch34_T20000"])
def test_in_run_covariance_matches_oracle(S, shape):
    """The proposal factor of an FP32 run at 65,536 particles (d = 14 and
    d = 23), as the run recorded it, equals the oracle's Cholesky factor of
    h^2 V with V the pooled covariance (divisor P - 1) of the particles
    entering that iteration: the first iteration of an M phase (covariance sums
    from the S-phase gather) and later ones (sums from the previous mutation
    launch's epilogue)."""
    w = I.WORKLOADS[shape]
    y = w.data()
    J, N = 64, 1024
    m = S.model_egarch(w.K, w.I, w.gamma)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=w.prior_seed)
    cfg = S.config_default(J=J, N=N, precision=S.FP32, seed=3)
    infos, design = _adaptive(S, m, cfg, y, th0)
    assert len(infos) >= 4
    starts = np.concatenate([[0], np.cumsum(design["R"])])
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP32, seed=3), y, th0)
    worst = 0.0
    late = len(infos) - 2
    for ell, r in ((1, 0), (1, 1), (2, 0), (2, 3), (late, 0), (late, 5)):
        th = _snapshot(ctx, th0, 3, design, ell, r)[0]
        _, V = O.mean_cov(th)
        Lg = design["L"][starts[ell - 1] + r]
        k, Lv = _h_tenths_of(Lg, V)
        assert 1 <= k <= 10
        # the recorded factor is h chol(V) for h a whole number of tenths
        Lo, z = O.cholesky((k / 10.0) ** 2 * V)
        assert z == 0
        err = _row_scaled_err(Lg, Lo)
        worst = max(worst, err)
        assert err < 1e-5, (ell, r, err)
        # and the covariance it implies
        Vg = Lg @ Lg.T / (k / 10.0) ** 2
        s = np.sqrt(np.diag(V))
        assert float((np.abs(Vg - V) / np.outer(s, s)).max()) < 1e-5, (ell, r)
    ctx.close()
    print(f"{shape}: worst row-scaled factor error {worst:.2e}")


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_step_size_and_iteration_rules_follow_the_paper(S, tempering):
    """Every iteration of an FP32 EGARCH(2,2) run: the step size h_r (in tenths)
    that the recorded factor carries starts at h0 = 0.5 and moves one tenth up
    when the iteration's pooled acceptance rate exceeds 0.25 and one down
    otherwise, clamped to [0.1, 1], carried across cycles; each cycle's mean
    acceptance rate is the mean of its iterations'; R_l = kappa Rbar when the
    cycle's RSS is below D2, else Rbar (Section 3.3, "Metropolis steps" and
    "M phase Termination")."""
    truth = I.WORKLOADS["egarch22_T5000"].truth
    y = I.simulate_egarch(truth, 1000, seed=8)
    J, N = 8, 512
    m = S.model_egarch(2, 2, True)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=21)
    tm = S.POWER if tempering == "power" else S.DATA
    cfg = S.config_default(J=J, N=N, precision=S.FP32, seed=9, tempering=tm)
    infos, design = _adaptive(S, m, cfg, y, th0)
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP32, seed=9, tempering=tm), y, th0)
    h = cfg.h0_tenths
    it = 0
    saw_up = saw_down = False
    for ell, info in enumerate(infos, start=1):
        R = int(design["R"][ell - 1])
        assert R == info["R"]
        assert R == (cfg.kappa * cfg.rbar if info["rss"] < cfg.d2 else cfg.rbar), (ell, info)
        snaps = [_snapshot(ctx, th0, 9, design, ell, r)[0] for r in range(R + 1)]
        accs = []
        for r in range(R):
            _, V = O.mean_cov(snaps[r])
            k, _ = _h_tenths_of(design["L"][it], V)
            assert k == h, (ell, r, k, h)
            acc = float(np.any(snaps[r + 1] != snaps[r], axis=1).mean())
            accs.append(acc)
            h_next = min(cfg.hmax_tenths, max(cfg.hmin_tenths, h + (1 if acc > cfg.acc_target else -1)))
            saw_up |= h_next > h
            saw_down |= h_next < h
            h = h_next
            it += 1
        assert info["h_tenths"] == h
        assert info["acc_rate"] == pytest.approx(np.mean(accs), abs=1e-12)
    ctx.close()
    assert saw_up and saw_down


def test_rne_stopping_rule_follows_the_paper(S):
    """RNE rule (Section 3.3, "M phase Termination"): each M phase stops after
    the first iteration at which the mean relative numerical efficiency of the
    test functions g1, g2, g3 (Section 5.2), computed by the oracle from the
    particles and their recursion states, reaches E1 (E2 in the last cycle,
    which ends at the full posterior), or at Rmax."""
    w = I.WORKLOADS["egarch11_T500"]
    y = w.data()
    J, N = 8, 256
    m = S.model_egarch(1, 1, False)
    spec = O.ModelSpec(K=1, I=1, gamma=False)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=w.prior_seed)
    kw = dict(J=J, N=N, precision=S.FP64, seed=4, rmax=40)
    infos, design = _adaptive(S, m, S.config_default(stop_rule=S.STOP_RNE, **kw), y, th0)
    cfg = S.config_default(stop_rule=S.STOP_RNE, **kw)
    ctx = S.init(m, S.config_default(**kw), y, th0)
    checked = 0
    for ell, info in enumerate(infos, start=1):
        R = int(design["R"][ell - 1])
        E = cfg.e2 if ell == len(infos) else cfg.e1
        for r in range(1, R + 1):
            th, _, _, st = _snapshot(ctx, th0, 4, design, ell, r)
            g = O.testfn(spec, th, st)
            rne = np.mean([O.moment(g[:, f], J, N)[3] for f in range(3)])
            if abs(rne - E) < 1e-9:
                continue   # a tie at rounding level decides nothing
            if r < R:
                assert rne < E, (ell, r, rne, E)
            else:
                assert rne >= E or R == cfg.rmax, (ell, r, rne, E)
            checked += 1
    ctx.close()
    assert checked >= len(infos)
