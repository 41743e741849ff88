"""Helpers for the GPU parity tests: seeded inputs and device buffers."""
import math

import numpy as np

from paper_1304_4334_gb300 import inputs as I


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a, dtype=None):
    torch = torch_cuda()
    dtype = dtype or torch.float64
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def soa(theta):
    """[P][d] host -> [d][P] float64 device."""
    return dev(np.ascontiguousarray(np.asarray(theta, float).T))


def host(t):
    return t.detach().cpu().numpy()


def egarch_truth(K, I_):
    """A process of the requested shape with about 1% daily volatility."""
    if I_ == 1:
        p, mu, sg = (1.0,), (0.0,), (1.0,)
    else:
        w = np.linspace(1.0, 0.3, I_)
        p, mu, sg = I.normalized_mixture(w, np.linspace(-0.2, 0.3, I_), np.linspace(0.8, 2.5, I_))
    alpha = tuple(np.linspace(0.97, 0.6, K))
    beta = tuple(np.linspace(0.08, 0.15, K))
    gamma = tuple(np.linspace(-0.05, 0.01, K))
    return I.EgarchTruth(0.0003, 0.01, alpha, beta, gamma, p, mu, sg)


def particles(spec_d, truth, K, I_, gamma, P, seed, prior=None, frac_prior=0.0):
    """Posterior-like cloud around the truth, optionally mixed with prior draws."""
    th = I.theta_of_truth(truth, I_model=I_, gamma=gamma)
    cloud = I.posterior_cloud(th, P, 0.05, seed)
    if prior is not None and frac_prior > 0:
        n = int(P * frac_prior)
        cloud[:n] = I.draw_prior(*prior, n, seed + 1)
    return cloud
