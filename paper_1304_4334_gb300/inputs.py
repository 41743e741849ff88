"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module generates inputs only.  It holds none of the simulator's arithmetic
(no likelihood, no weights, no resampling): it simulates returns forward from the
EGARCH data-generating process (eqs. EGARCH_mod1, EGARCH_mod2 and the normal
mixture of Section 5.1), draws particles from a Gaussian prior, and builds
regression data for the conjugate check.  All randomness is numpy PCG64 with the
stated seed.  The S&P 500 series of Section 5 is not available, so these stand in
for it: daily-return-like data with about 1% volatility.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)


@dataclass
class EgarchTruth:
    """Model-space parameters of a data-generating process."""
    mu_y: float
    sigma_y: float
    alpha: tuple
    beta: tuple
    gamma: tuple
    p: tuple = (1.0,)
    mu: tuple = (0.0,)
    sig: tuple = (1.0,)

    @property
    def K(self):
        return len(self.alpha)

    @property
    def I(self):
        return len(self.p)


def normalized_mixture(p, mu_raw, sd_raw):
    """Center and scale a raw normal mixture so that E eps = 0 and var eps = 1."""
    p = np.asarray(p, float) / np.sum(p)
    mu_raw = np.asarray(mu_raw, float)
    sd_raw = np.asarray(sd_raw, float)
    m = np.sum(p * mu_raw)
    mu_c = mu_raw - m
    scale = 1.0 / math.sqrt(np.sum(p * (mu_c ** 2 + sd_raw ** 2)))
    return tuple(p), tuple(mu_c * scale), tuple(sd_raw * scale)


def simulate_egarch(truth: EgarchTruth, T: int, seed: int, return_path=False):
    """Simulate y_1..y_T forward from the EGARCH(K, I) process.

    v_k0 = 0 and no shock precedes the first observation (v_k1 = 0); then
    v_kt = alpha_k v_k,t-1 + beta_k (|eps_t-1| - (2/pi)^1/2) + gamma_k eps_t-1,
    y_t = mu_Y + sigma_Y exp(sum_k v_kt / 2) eps_t, eps_t from the mixture.
    With return_path the shocks eps_t, the volatilities h_t and h_{T+1} come back
    too (used to check the likelihood by inversion)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K, I = truth.K, truth.I
    comp = rng.choice(I, size=T, p=np.asarray(truth.p) / np.sum(truth.p))
    z = rng.standard_normal(T)
    eps = np.asarray(truth.mu)[comp] + np.asarray(truth.sig)[comp] * z
    alpha = np.asarray(truth.alpha, float)
    beta = np.asarray(truth.beta, float)
    gamma = np.asarray(truth.gamma, float)
    v = np.zeros(K)
    y = np.empty(T)
    h = np.empty(T)
    for t in range(T):
        if t > 0:
            v = alpha * v + beta * (abs(eps[t - 1]) - SQRT_2_OVER_PI) + gamma * eps[t - 1]
        h[t] = truth.sigma_y * math.exp(0.5 * float(np.sum(v)))
        y[t] = truth.mu_y + h[t] * eps[t]
    if not return_path:
        return y
    v_next = alpha * v + beta * (abs(eps[-1]) - SQRT_2_OVER_PI) + gamma * eps[-1]
    h_next = truth.sigma_y * math.exp(0.5 * float(np.sum(v_next)))
    return y, eps, h, v.copy(), h_next


def theta_of_truth(truth: EgarchTruth, I_model=None, gamma=True):
    """Transformed parameter vector (Table 1 layout) that maps to ``truth``.

    Layout: theta_1, theta_2, theta_3k, theta_4k, [theta_5k], [theta_6i, theta_7i,
    theta_8i].  A model with more mixture components than the process gets the
    extra components at negligible weight."""
    I_model = truth.I if I_model is None else I_model
    th = [truth.mu_y * 1000.0, math.log(truth.sigma_y)]
    th += [math.atanh(a) for a in truth.alpha]
    th += [math.log(b) for b in truth.beta]
    if gamma:
        th += list(truth.gamma)
    if I_model >= 2:
        p = list(truth.p) + [1e-3] * (I_model - truth.I)
        mu = list(truth.mu) + [0.0] * (I_model - truth.I)
        sg = list(truth.sig) + [1.0] * (I_model - truth.I)
        p = np.asarray(p) / np.sum(p)
        th += [math.atanh(pi - 1.0) for pi in p]       # p*_i = p_i lies in (0, 2)
        th += list(mu)
        th += [math.log(s) for s in sg]
    return np.asarray(th)


def draw_prior(mean, sd, lo, P: int, seed: int):
    """P draws from independent normals N(mean_i, sd_i^2) truncated below at lo_i
    (rejection), row-major [P][d]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mean, sd, lo = (np.asarray(a, float) for a in (mean, sd, lo))
    d = len(mean)
    out = np.empty((P, d))
    for i in range(d):
        col = mean[i] + sd[i] * rng.standard_normal(P)
        bad = col < lo[i]
        while np.any(bad):
            col[bad] = mean[i] + sd[i] * rng.standard_normal(int(bad.sum()))
            bad = col < lo[i]
        out[:, i] = col
    return out


def posterior_cloud(theta_true, P: int, scale: float, seed: int):
    """theta_true + N(0, scale^2) per component: a posterior-like particle cloud."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.asarray(theta_true, float)
    return t[None, :] + scale * rng.standard_normal((P, len(t)))


def linreg_data(T: int, beta, sigma: float, seed: int):
    """X ~ N(0,1) iid, y = X beta + N(0, sigma^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beta = np.asarray(beta, float)
    X = rng.standard_normal((T, len(beta)))
    y = X @ beta + sigma * rng.standard_normal(T)
    return X, y


# ---------------------------------------------------------------------------------
# Workloads.  Shapes follow Section 5 (J = 64 groups of N = 1024, T about 5000
# daily returns at about 1% volatility) scaled as listed.
# ---------------------------------------------------------------------------------
def _truth_k2_i2():
    p, mu, sg = normalized_mixture((0.8, 0.2), (0.0, 0.0), (1.0, 2.5))
    return EgarchTruth(mu_y=0.0003, sigma_y=0.01, alpha=(0.98, 0.85), beta=(0.10, 0.15),
                       gamma=(-0.05, 0.0), p=p, mu=mu, sig=sg)


def _truth_k3_heavy_tails():
    p, mu, sg = normalized_mixture((0.9, 0.1), (0.0, 0.0), (1.0, 4.0))
    return EgarchTruth(mu_y=0.0003, sigma_y=0.01, alpha=(0.98, 0.90, 0.60),
                       beta=(0.08, 0.10, 0.12), gamma=(-0.04, -0.02, 0.0), p=p, mu=mu, sig=sg)


@dataclass
class Workload:
    name: str
    K: int
    I: int
    gamma: bool
    T: int
    J: int
    N: int
    precision: str          # "f64" or "f32"
    mutation: str           # "rw" or "mala"
    truth: EgarchTruth
    data_seed: int
    prior_seed: int
    rbar: int = 7
    kappa: int = 3
    extra: dict = field(default_factory=dict)

    @property
    def P(self):
        return self.J * self.N

    def data(self):
        return simulate_egarch(self.truth, self.T, self.data_seed)


WORKLOADS = {
    # EGARCH(1,1), Gaussian shocks, no leverage term: 4 parameters.  The stated
    # (omega, alpha, beta) = (-0.1, 0.1, 0.98) of log h^2 = omega + b log h^2_{t-1} +
    # a(|eps|-c) maps to alpha_1 = 0.98, beta_1 = 0.1, sigma_Y = exp(omega/(2(1-b))).
    "egarch11_T500": Workload("egarch11_T500", 1, 1, False, 500, 4, 256, "f64", "rw",
                              EgarchTruth(0.0, math.exp(-0.1 / (2 * 0.02)), (0.98,), (0.1,), (0.0,)),
                              data_seed=11, prior_seed=12, rbar=10, kappa=1),
    "egarch22_T5000": Workload("egarch22_T5000", 2, 2, True, 5000, 64, 1024, "f32", "rw",
                               _truth_k2_i2(), data_seed=21, prior_seed=22),
    "egarch22_T5000_mala": Workload("egarch22_T5000_mala", 2, 2, True, 5000, 64, 4096, "f32",
                                    "mala", _truth_k2_i2(), data_seed=21, prior_seed=32),
    "egarch34_T20000": Workload("egarch34_T20000", 3, 4, True, 20000, 128, 8192, "f32", "rw",
                                _truth_k3_heavy_tails(), data_seed=51, prior_seed=52),
}


def batched_workloads(n: int = 32, seed: int = 40, J: int = 16, N: int = 1024):
    """n datasets with T ~ U{500..10000}, K ~ U{1,2,3}, I ~ U{1..4}; each dataset
    is simulated from a process of its own (K, I)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n):
        T = int(rng.integers(500, 10001))
        K = int(rng.integers(1, 4))
        I = int(rng.integers(1, 5))
        alpha = tuple(float(a) for a in np.sort(rng.uniform(0.5, 0.985, K))[::-1])
        beta = tuple(float(x) for x in rng.uniform(0.05, 0.15, K))
        gamma = tuple(float(x) for x in rng.uniform(-0.05, 0.02, K))
        if I == 1:
            p, mu, sg = (1.0,), (0.0,), (1.0,)
        else:
            w = rng.dirichlet(np.full(I, 3.0))
            p, mu, sg = normalized_mixture(w, rng.normal(0, 0.3, I), rng.uniform(0.7, 2.5, I))
        truth = EgarchTruth(0.0002, float(rng.uniform(0.007, 0.015)), alpha, beta, gamma, p, mu, sg)
        out.append(Workload(f"batch{b}", K, I, True, T, J, N, "f32", "rw", truth,
                            data_seed=1000 + b, prior_seed=2000 + b))
    return out
