"""Algorithm 3 (hybrid) on the GPU through the C ABI: the recorded design of an
adaptive run, replayed with the same seed, reproduces that run; replayed with a
new seed it gives estimates consistent with the conjugate closed form; and the
oracle replaying the GPU's design agrees with the GPU replay within NSE."""
import math

import numpy as np
import pytest
from scipy import stats

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


def _linreg():
    beta = np.array([0.5, -1.0, 2.0])
    X, y = I.linreg_data(60, beta, 1.0, seed=3)
    m0, s0 = np.zeros(3), np.full(3, 2.0)
    V0 = np.diag(s0 ** 2)
    lml = stats.multivariate_normal(X @ m0, np.eye(60) + X @ V0 @ X.T).logpdf(y)
    Vn = np.linalg.inv(np.linalg.inv(V0) + X.T @ X)
    return X, y, m0, s0, lml, Vn @ (X.T @ y), Vn


@pytest.mark.parametrize("tempering", ["power", "data"])
def test_hybrid_on_gpu(S, tempering):
    X, y, m0, s0, lml, mn, Vn = _linreg()
    J, N = 32, 256
    m = S.model_linreg(3, 1.0, m0, s0)
    tm = S.POWER if tempering == "power" else S.DATA
    th0 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=5)
    a = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, tempering=tm, seed=3), y, th0, X=X)
    a.record_design()
    a.run()
    design = a.design()
    lm_a = a.log_ml()
    th_a = a.particles()[0]
    a.close()
    assert len(design["x"]) >= 2 and design["L"].shape[0] == design["R"].sum()
    # same seed: the replay is the adaptive run
    b = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, tempering=tm, seed=3), y, th0, X=X)
    b.replay_design(design)
    b.run()
    assert b.log_ml()[0] == pytest.approx(lm_a[0], abs=1e-9)
    np.testing.assert_allclose(b.particles()[0], th_a, rtol=0, atol=1e-12)
    b.close()
    # new seed and prior draws (Algorithm 3, step 2)
    th1 = I.draw_prior(m0, s0, np.full(3, -np.inf), J * N, seed=6)
    c = S.init(m, S.config_default(J=J, N=N, precision=S.FP64, tempering=tm, seed=99), y, th1, X=X)
    c.replay_design(design)
    n, info = c.run()
    assert n == len(design["x"]) and info["done"] == 1
    lm, nse, _ = c.log_ml()
    mom = c.moments()
    c.close()
    assert abs(lm - lml) < 3 * nse, (lm, lml, nse)
    for i in range(3):
        assert abs(mom[i, 0] - mn[i]) < 3 * mom[i, 2]
    # the oracle replaying the GPU's design
    spec = O.ModelSpec(model=O.LINREG, p=3, sigma=1.0, prior_mean=m0, prior_sd=s0)
    r = O.smc_run(spec, y, th1, J, N, X=X, tempering=1 if tempering == "power" else 0, seed=99,
                  design=design)
    assert r["status"] == 0 and r["cycles"] == len(design["x"])
    assert abs(r["log_ml"] - lm) < 3 * math.hypot(r["log_ml_nse"], nse)
