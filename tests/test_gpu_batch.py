"""Batched runs (many datasets of different T and EGARCH (K, I) advanced
together, one persistent M-phase kernel per Metropolis iteration) must give
the same particles and estimates as the same runs done one at a time: the
kernels, the counter-addressed random numbers and the reductions are the
same, so the comparison is exact up to nothing."""
import numpy as np
import pytest

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


def _members(S, n, J, N, seed):
    ws = I.batched_workloads(n=n, seed=seed, J=J, N=N)
    models, cfgs, ys, ths = [], [], [], []
    for k, w in enumerate(ws):
        m = S.model_egarch(w.K, w.I, True)
        mean, sd, lo = S.model_prior(m)
        models.append(m)
        cfgs.append(S.config_default(J=J, N=N, precision=S.FP32, seed=100 + k))
        ys.append(I.simulate_egarch(w.truth, min(w.T, 1500), seed=w.data_seed))
        ths.append(I.draw_prior(mean, sd, lo, J * N, seed=w.prior_seed))
    return ws, models, cfgs, ys, ths


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_individual_runs(S, autotune):
    ws, models, cfgs, ys, ths = _members(S, 5, 4, 96, seed=7)
    b = S.Batch(models, cfgs, ys, ths)
    if autotune:
        b.autotune(iters=1)
        assert b.tile in (64, 128, 256)
    ncyc = b.run()
    assert ncyc >= 1
    for i in range(len(models)):
        ctx = S.init(models[i], cfgs[i], ys[i], ths[i])
        ctx.run()
        lm1, nse1, lt1 = ctx.log_ml()
        th1, ll1, lp1, _ = ctx.particles()
        mem = b.member(i)
        lm2, nse2, lt2 = mem.log_ml()
        th2, ll2, lp2, _ = mem.particles()
        ctx.close()
        assert lm1 == lm2 and nse1 == nse2 and lt1 == lt2, (i, lm1, lm2)
        np.testing.assert_array_equal(th1, th2)
        np.testing.assert_array_equal(ll1, ll2)
    e, ms, cy = b.totals()
    assert e > 0 and ms > 0 and cy == ncyc
    b.close()


def test_batch_of_uneven_lengths_and_models_runs_to_the_posterior(S):
    ws, models, cfgs, ys, ths = _members(S, 12, 4, 128, seed=11)
    b = S.Batch(models, cfgs, ys, ths)
    b.autotune(iters=1)
    b.run()
    for i in range(len(models)):
        lm, nse, lt = b.member(i).log_ml()
        assert np.isfinite(lm) and 0 <= nse < 5
        _, _, _, st = b.member(i).particles()
    b.close()
