"""Whole FP32 runs of the K >= 2 EGARCH models against whole oracle runs.

These runs have no closed form: the GPU's FP32 run (FP32 recursion, FP64
accumulators) and the oracle's FP64 run of the same data from the same prior
draws are independent Monte Carlo estimates of the same posterior, so their
log marginal likelihoods and posterior means must agree within 3 combined
numerical standard errors (Algorithm 2 and Section 4.2; Proposition 1 for the
NSE).  J = 32 groups, so that each NSE rests on 31 degrees of freedom.
The model shapes are those of the benchmark workloads (K = 2, I = 2 and
K = 3, I = 4), on the first T = 5000 observations of their synthetic series.
"""
import math
import os

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


@pytest.mark.parametrize("shape", ["egarch22_T5000", "egarch34_T20000"])
def test_fp32_run_agrees_with_oracle_run(S, shape):
    w = I.WORKLOADS[shape]
    y = w.data()[:5000]
    J, N = 32, 128
    m = S.model_egarch(w.K, w.I, w.gamma)
    mean, sd, lo = S.model_prior(m)
    th0 = I.draw_prior(mean, sd, lo, J * N, seed=w.prior_seed + 7)
    ctx = S.init(m, S.config_default(J=J, N=N, precision=S.FP32, seed=31), y, th0)
    ctx.run()
    lm, nse, _ = ctx.log_ml()
    th_g = ctx.particles()[0]
    ctx.close()
    spec = O.ModelSpec(K=w.K, I=w.I, gamma=w.gamma)
    r = O.smc_run(spec, y, th0, J, N, seed=1031, nthreads=os.cpu_count() or 4)
    assert r["status"] == 0
    comb = math.hypot(nse, r["log_ml_nse"])
    print(f"{shape}: log ML GPU {lm:.4f} +- {nse:.4f}, oracle {r['log_ml']:.4f} +- {r['log_ml_nse']:.4f}, "
          f"difference {abs(lm - r['log_ml']) / comb:.2f} combined NSE")
    assert abs(lm - r["log_ml"]) < 3 * comb
    worst = 0.0
    for i in range(spec.d):
        mg, _, ng, _ = O.moment(th_g[:, i], J, N)
        mo, _, no, _ = O.moment(r["theta"][:, i], J, N)
        z = abs(mg - mo) / math.hypot(ng, no)
        worst = max(worst, z)
        assert z < 3, (i, mg, mo, ng, no)
    print(f"{shape}: largest posterior-mean difference {worst:.2f} combined NSE over {spec.d} parameters")


def test_fp32_loglik_at_the_largest_shape(S):
    """FP32 log likelihood of the K = 3, I = 4 model over all T = 20000
    observations against the FP64 oracle, for posterior-like particles:
    1e-6 relative (7e-8 measured; the FP32 tolerance is 1e-4)."""
    torch = torch_cuda()
    w = I.WORKLOADS["egarch34_T20000"]
    y = w.data()
    spec = O.ModelSpec(K=w.K, I=w.I, gamma=w.gamma)
    th = I.posterior_cloud(I.theta_of_truth(w.truth, I_model=w.I, gamma=w.gamma), 333, 0.05, seed=3)
    ll_o = O.loglik(spec, y, th, nthreads=os.cpu_count() or 4)
    m = S.model_egarch(w.K, w.I, w.gamma)
    ll = torch.empty(333, dtype=torch.float64, device="cuda")
    theta = torch.as_tensor(np.ascontiguousarray(th.T), device="cuda")
    S.loglik(m, S.FP32, torch.as_tensor(y, dtype=torch.float32, device="cuda"), theta, ll)
    torch.cuda.synchronize()
    ll = ll.cpu().numpy()
    rel = np.abs(ll - ll_o) / np.abs(ll_o)
    print(f"K=3, I=4, T=20000 FP32 log likelihood: max rel {rel.max():.2e}, median {np.median(rel):.2e}")
    np.testing.assert_allclose(ll, ll_o, rtol=1e-6)
    # the mutation kernel's recursion (alpha v as one FMA): a step with a zero
    # proposal factor from a current log likelihood of -inf accepts theta itself
    # and stores its log likelihood
    d = spec.d
    llm = torch.full((333,), -math.inf, dtype=torch.float64, device="cuda")
    lpm = torch.as_tensor(O.logprior(spec, th), device="cuda")
    tm = theta.clone()
    n = S.mutate_rw(m, S.FP32, torch.as_tensor(y, dtype=torch.float32, device="cuda"), tm, llm, lpm, None,
                    torch.zeros((d, d), dtype=torch.float64, device="cuda"), 1.0, 5, 1, 0)
    assert n == 333
    np.testing.assert_array_equal(tm.cpu().numpy(), theta.cpu().numpy())
    llm = llm.cpu().numpy()
    relm = np.abs(llm - ll_o) / np.abs(ll_o)
    print(f"  mutation kernel: max rel {relm.max():.2e}, median {np.median(relm):.2e}")
    np.testing.assert_allclose(llm, ll_o, rtol=1e-6)
