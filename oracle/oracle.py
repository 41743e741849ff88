"""ctypes binding of the C oracle (``oracle/*.c``), plus its build step.

TEST INFRASTRUCTURE ONLY.  Argument marshalling; all arithmetic is in the C
sources, which follow the paper passage by passage (see their headers).
Arrays are numpy float64, particle-major ([P][d]).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["philox.c", "model.c", "smc.c"]
_lock = threading.Lock()
_lib = None

EGARCH, LINREG = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc (host arch)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", _SO + ".tmp"] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_SO)
            _declare(_lib)
    return _lib


dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)
i32p = C.POINTER(C.c_int32)
u64p = C.POINTER(C.c_uint64)


class Model(C.Structure):
    _fields_ = [("model", C.c_int), ("K", C.c_int), ("I", C.c_int), ("gamma", C.c_int),
                ("p", C.c_int), ("sigma", C.c_double), ("d_full", C.c_int), ("d", C.c_int),
                ("free_idx", ip), ("theta_fixed", dp), ("prior_mean", dp),
                ("prior_sd", dp), ("prior_lo", dp), ("eps0_zero", C.c_int)]


class EgarchPar(C.Structure):
    _fields_ = [("mu_y", C.c_double), ("sigma_y", C.c_double),
                ("alpha", C.c_double * 8), ("beta", C.c_double * 8), ("gamma", C.c_double * 8),
                ("p", C.c_double * 8), ("mu", C.c_double * 8), ("sig", C.c_double * 8)]


class RunCfg(C.Structure):
    _fields_ = [("J", C.c_int), ("N", C.c_int), ("tempering", C.c_int), ("mutation", C.c_int),
                ("resid", C.c_int), ("d1", C.c_double), ("d2", C.c_double),
                ("stop_rule", C.c_int), ("rbar", C.c_int), ("kappa", C.c_int), ("rmax", C.c_int),
                ("e1", C.c_double), ("e2", C.c_double), ("h0_tenths", C.c_int),
                ("hmin_tenths", C.c_int), ("hmax_tenths", C.c_int), ("acc_target", C.c_double),
                ("h_reset_each_cycle", C.c_int), ("force_dates", ip), ("n_force", C.c_int),
                ("bisect_iters", C.c_int), ("seed", C.c_uint64), ("max_cycles", C.c_int),
                ("nthreads", C.c_int), ("replay", C.c_int), ("n_design", C.c_int),
                ("design_x", dp), ("design_R", ip), ("design_L", dp), ("rec_L", dp),
                ("rec_L_cap", C.c_int), ("burnin", C.c_int), ("pit_out", dp)]


class RunOut(C.Structure):
    _fields_ = [("cycles", C.c_int), ("metropolis_steps", C.c_long),
                ("particle_obs_evals", C.c_double), ("log_ml", C.c_double),
                ("log_ml_nse", C.c_double), ("log_ml_tilde", C.c_double),
                ("h_final_tenths", C.c_int), ("status", C.c_int),
                ("log_score", C.c_double), ("log_score_nse", C.c_double)]


def _declare(L):
    L.or_philox4x64.argtypes = [u64p, u64p, u64p]
    L.or_philox_normals.argtypes = [C.c_uint64] * 4 + [C.c_int, dp]
    L.or_philox_log_uniform.argtypes = [C.c_uint64] * 4
    L.or_philox_log_uniform.restype = C.c_double
    L.or_egarch_dim.argtypes = [C.c_int] * 3
    L.or_egarch_dim.restype = C.c_int
    L.or_egarch_prior_table1.argtypes = [C.c_int] * 3 + [dp] * 3
    L.or_egarch_transform.argtypes = [C.c_int] * 3 + [dp, C.POINTER(EgarchPar)]
    L.or_logprior.argtypes = [C.POINTER(Model), dp]
    L.or_logprior.restype = C.c_double
    L.or_loglik.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp]
    L.or_loglik.restype = C.c_double
    L.or_loglik_range.argtypes = [C.POINTER(Model), dp, dp, C.c_int, C.c_int, dp, dp]
    L.or_loglik_range.restype = C.c_double
    L.or_loglik_terms.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp]
    L.or_loglik_grad.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp]
    L.or_loglik_grad.restype = C.c_double
    L.or_logprior_grad.argtypes = [C.POINTER(Model), dp, dp]
    L.or_egarch_testfn.argtypes = [C.POINTER(Model), dp, dp, dp]
    L.or_loglik_batch.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, C.c_int, dp, dp, C.c_int]
    L.or_logprior_batch.argtypes = [C.POINTER(Model), dp, C.c_int, dp]
    L.or_moment.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp, dp]
    L.or_ess_log.argtypes = [dp, C.c_int]
    L.or_ess_log.restype = C.c_double
    L.or_log_ml.argtypes = [dp, C.c_int, dp, dp]
    L.or_resample.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, i32p]
    L.or_resample.restype = C.c_int
    L.or_resample_scheme.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, i32p]
    L.or_resample_scheme.restype = C.c_int
    L.or_mean_cov.argtypes = [dp, C.c_int, C.c_int, dp, dp]
    L.or_cholesky.argtypes = [dp, C.c_int, dp]
    L.or_cholesky.restype = C.c_int
    L.or_mutate_rw.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp, dp, dp, C.c_int, dp,
                               C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, ip, C.c_int]
    L.or_mutate_rw.restype = C.c_long
    L.or_mutate_mala.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp, dp, dp, dp, C.c_int,
                                 dp, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, ip, C.c_int]
    L.or_mutate_mala.restype = C.c_long
    L.or_mutate_indep.argtypes = [C.POINTER(Model), dp, dp, C.c_int, dp, dp, dp, dp, C.c_int, dp, dp,
                                  C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, ip, C.c_int]
    L.or_mutate_indep.restype = C.c_long
    L.or_draw_prior.argtypes = [C.POINTER(Model), C.c_uint64, C.c_int, dp]
    L.or_pit_shock.argtypes = [C.POINTER(Model), dp, C.c_uint64, C.c_uint64, C.c_int]
    L.or_pit_shock.restype = C.c_double
    L.or_power_search.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_int, dp]
    L.or_power_search.restype = C.c_double
    L.or_smc_run.argtypes = [C.POINTER(Model), dp, dp, C.c_int, C.POINTER(RunCfg), dp, dp, dp,
                             dp, dp, dp, ip, dp, ip, dp, C.POINTER(RunOut)]
    L.or_smc_run.restype = C.c_int


def _d(a):
    return a.ctypes.data_as(dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------------
class ModelSpec:
    """Model description.  Keeps the numpy buffers the C struct points into alive."""

    def __init__(self, model=EGARCH, K=1, I=1, gamma=True, p=0, sigma=1.0,
                 prior_mean=None, prior_sd=None, prior_lo=None,
                 free_idx=None, theta_fixed=None, eps0_zero=False):
        L = _load()
        self.model, self.K, self.I, self.gamma, self.p, self.sigma = model, K, I, bool(gamma), p, sigma
        if model == EGARCH:
            d_full = L.or_egarch_dim(K, I, int(gamma))
        else:
            d_full = p
        self.d_full = d_full
        if prior_mean is None:
            assert model == EGARCH
            pm, ps, pl = table1_prior(K, I, gamma)
        else:
            pm, ps, pl = prior_mean, prior_sd, prior_lo
            if pl is None:
                pl = np.full(len(pm), -np.inf)
        if free_idx is not None:
            self.free_idx = np.ascontiguousarray(free_idx, dtype=np.int32)
            self.theta_fixed = _f64(theta_fixed)
            d = len(self.free_idx)
            if len(pm) == d_full:
                pm, ps, pl = (np.asarray(x)[self.free_idx] for x in (pm, ps, pl))
        else:
            self.free_idx, self.theta_fixed, d = None, None, d_full
        self.d = d
        self.prior_mean, self.prior_sd, self.prior_lo = _f64(pm), _f64(ps), _f64(pl)
        assert len(self.prior_mean) == d
        self.eps0_zero = eps0_zero
        self.c = Model(model, K, I, int(gamma), p, sigma, d_full, d,
                       self.free_idx.ctypes.data_as(ip) if self.free_idx is not None else None,
                       _d(self.theta_fixed), _d(self.prior_mean), _d(self.prior_sd),
                       _d(self.prior_lo), int(eps0_zero))

    @property
    def nstate(self):
        return self.K + 1 if self.model == EGARCH else 1


def table1_prior(K, I, gamma=True):
    L = _load()
    d = L.or_egarch_dim(K, I, int(gamma))
    m, s, lo = (np.zeros(d) for _ in range(3))
    L.or_egarch_prior_table1(K, I, int(gamma), _d(m), _d(s), _d(lo))
    return m, s, lo


def egarch_dim(K, I, gamma=True):
    return _load().or_egarch_dim(K, I, int(gamma))


def philox4x64(ctr, key):
    L = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    L.or_philox4x64(c.ctypes.data_as(u64p), k.ctypes.data_as(u64p), out.ctypes.data_as(u64p))
    return out


def philox_normals(seed, p, it, cycle, d):
    z = np.zeros(d)
    _load().or_philox_normals(seed, p, it, cycle, d, _d(z))
    return z


def philox_log_uniform(seed, p, it, cycle):
    return _load().or_philox_log_uniform(seed, p, it, cycle)


def egarch_transform(K, I, gamma, theta_full):
    L = _load()
    q = EgarchPar()
    L.or_egarch_transform(K, I, int(gamma), _d(_f64(theta_full)), C.byref(q))
    return dict(mu_y=q.mu_y, sigma_y=q.sigma_y, alpha=np.array(q.alpha[:K]),
                beta=np.array(q.beta[:K]), gamma=np.array(q.gamma[:K]),
                p=np.array(q.p[:I]), mu=np.array(q.mu[:I]), sig=np.array(q.sig[:I]))


def logprior(spec, theta):
    theta = _f64(np.atleast_2d(theta))
    out = np.zeros(theta.shape[0])
    _load().or_logprior_batch(C.byref(spec.c), _d(theta), theta.shape[0], _d(out))
    return out


def loglik(spec, y, theta, X=None, nthreads=1, with_state=False):
    theta = _f64(np.atleast_2d(theta))
    y = _f64(y)
    Xa = _f64(X) if X is not None else None
    P = theta.shape[0]
    out = np.zeros(P)
    st = np.zeros((P, spec.nstate))
    _load().or_loglik_batch(C.byref(spec.c), _d(y), _d(Xa), len(y), _d(theta), P, _d(out),
                            _d(st), nthreads)
    return (out, st) if with_state else out


def loglik_range(spec, y, t0, t1, theta, state, X=None):
    """Continue one particle's recursion from ``state`` at t0 through t1 (in place)."""
    st = _f64(state).copy()
    v = _load().or_loglik_range(C.byref(spec.c), _d(_f64(y)), _d(_f64(X) if X is not None else None),
                                t0, t1, _d(_f64(theta)), _d(st))
    return v, st


def loglik_terms(spec, y, theta, X=None):
    y = _f64(y)
    out = np.zeros(len(y))
    _load().or_loglik_terms(C.byref(spec.c), _d(y), _d(_f64(X) if X is not None else None),
                            len(y), _d(_f64(theta)), _d(out))
    return out


def loglik_grad(spec, y, theta, X=None):
    theta = _f64(np.atleast_2d(theta))
    y = _f64(y)
    Xa = _f64(X) if X is not None else None
    P = theta.shape[0]
    g = np.zeros((P, spec.d))
    ll = np.zeros(P)
    L = _load()
    for n in range(P):
        row = np.ascontiguousarray(theta[n])
        gn = np.zeros(spec.d)
        ll[n] = L.or_loglik_grad(C.byref(spec.c), _d(y), _d(Xa), len(y), _d(row), _d(gn))
        g[n] = gn
    return ll, g


def logprior_grad(spec, theta):
    theta = _f64(np.atleast_2d(theta))
    g = np.zeros_like(theta)
    L = _load()
    for n in range(theta.shape[0]):
        row = np.ascontiguousarray(theta[n])
        gn = np.zeros(spec.d)
        L.or_logprior_grad(C.byref(spec.c), _d(row), _d(gn))
        g[n] = gn
    return g


def testfn(spec, theta, state):
    theta = _f64(np.atleast_2d(theta))
    state = _f64(np.atleast_2d(state))
    out = np.zeros((theta.shape[0], 3))
    L = _load()
    for n in range(theta.shape[0]):
        g = np.zeros(3)
        L.or_egarch_testfn(C.byref(spec.c), _d(np.ascontiguousarray(theta[n])),
                           _d(np.ascontiguousarray(state[n])), _d(g))
        out[n] = g
    return out


def moment(g, J, N):
    g = _f64(g)
    r = [C.c_double() for _ in range(4)]
    _load().or_moment(_d(g), J, N, *[C.byref(x) for x in r])
    return tuple(x.value for x in r)   # mean, sd, nse, rne


def ess_log(logw):
    logw = _f64(logw)
    return _load().or_ess_log(_d(logw), len(logw))


def log_ml(a):
    a = _f64(a)
    x, s = C.c_double(), C.c_double()
    _load().or_log_ml(_d(a), len(a), C.byref(x), C.byref(s))
    return x.value, s.value


def resample(w, J, N, resid=True, seed=0, cycle=0):
    w = _f64(w)
    idx = np.zeros(J * N, dtype=np.int32)
    st = _load().or_resample(_d(w), J, N, int(resid), seed, cycle, idx.ctypes.data_as(i32p))
    if st != 0:
        raise ValueError("degenerate group (all weights zero)")
    return idx.reshape(J, N)


RESIDUAL, MULTINOMIAL, STRATIFIED, SYSTEMATIC = 0, 1, 2, 3
RW, MALA, INDEP = 0, 1, 2


def resample_scheme(w, J, N, scheme, seed=0, cycle=0):
    w = _f64(w)
    idx = np.zeros(J * N, dtype=np.int32)
    st = _load().or_resample_scheme(_d(w), J, N, scheme, seed, cycle, idx.ctypes.data_as(i32p))
    if st != 0:
        raise ValueError("degenerate group (all weights zero)")
    return idx.reshape(J, N)


def mean_cov(theta):
    theta = _f64(theta)
    P, d = theta.shape
    m = np.zeros(d)
    c = np.zeros((d, d))
    _load().or_mean_cov(_d(theta), P, d, _d(m), _d(c))
    return m, c


def cholesky(A):
    A = _f64(A)
    d = A.shape[0]
    Lm = np.zeros((d, d))
    z = _load().or_cholesky(_d(A), d, _d(Lm))
    return Lm, z


def mutate_rw(spec, y, theta, ll, lp, state, Lmat, phi, seed, cycle, it, X=None, nthreads=1):
    """One random-walk Metropolis step, in place on copies; returns new arrays."""
    theta = _f64(theta).copy(); ll = _f64(ll).copy(); lp = _f64(lp).copy()
    state = _f64(state).copy()
    P = theta.shape[0]
    acc = np.zeros(P, dtype=np.int32)
    n = _load().or_mutate_rw(C.byref(spec.c), _d(_f64(y)), _d(_f64(X) if X is not None else None),
                             len(y), _d(theta), _d(ll), _d(lp), _d(state), P, _d(_f64(Lmat)),
                             phi, seed, cycle, it, acc.ctypes.data_as(ip), nthreads)
    return theta, ll, lp, state, acc, n


def mutate_indep(spec, y, theta, ll, lp, state, mbar, Lmat, phi, seed, cycle, it, X=None, nthreads=1):
    """One independent Gaussian Metropolis step with proposal N(mbar, L L^T)
    (Section 3.3's alternative sampler); returns new arrays."""
    theta = _f64(theta).copy(); ll = _f64(ll).copy(); lp = _f64(lp).copy()
    state = _f64(state).copy()
    P = theta.shape[0]
    acc = np.zeros(P, dtype=np.int32)
    n = _load().or_mutate_indep(C.byref(spec.c), _d(_f64(y)), _d(_f64(X) if X is not None else None),
                                len(y), _d(theta), _d(ll), _d(lp), _d(state), P, _d(_f64(mbar)),
                                _d(_f64(Lmat)), phi, seed, cycle, it, acc.ctypes.data_as(ip), nthreads)
    return theta, ll, lp, state, acc, n


def mutate_mala(spec, y, theta, ll, lp, grad, state, Lmat, phi, seed, cycle, it, X=None,
                nthreads=1):
    theta = _f64(theta).copy(); ll = _f64(ll).copy(); lp = _f64(lp).copy()
    grad = _f64(grad).copy(); state = _f64(state).copy()
    P = theta.shape[0]
    acc = np.zeros(P, dtype=np.int32)
    n = _load().or_mutate_mala(C.byref(spec.c), _d(_f64(y)), _d(_f64(X) if X is not None else None),
                               len(y), _d(theta), _d(ll), _d(lp), _d(grad), _d(state), P,
                               _d(_f64(Lmat)), phi, seed, cycle, it, acc.ctypes.data_as(ip), nthreads)
    return theta, ll, lp, grad, state, acc, n


def draw_prior(spec, seed, P):
    """Prior draws theta[P][d] from Table 1 by Philox (truncation by rejection)."""
    th = np.zeros((P, spec.d))
    _load().or_draw_prior(C.byref(spec.c), seed, P, _d(th))
    return th


def pit_shock(spec, theta, seed, particle, s):
    """Simulated standardized shock of the PIT draw Y_s (Section 4.1)."""
    return _load().or_pit_shock(C.byref(spec.c), _d(_f64(theta)), seed, particle, s)


def power_search(ll, phi, d1=0.5, iters=60):
    ll = _f64(ll)
    r = C.c_double()
    dphi = _load().or_power_search(_d(ll), len(ll), phi, d1, iters, C.byref(r))
    return dphi, r.value


DEFAULT_RUN = dict(tempering=1, mutation=0, resid=1, d1=0.5, d2=0.2, stop_rule=0, rbar=7,
                   kappa=3, rmax=100, e1=0.35, e2=0.90, h0_tenths=5, hmin_tenths=1,
                   hmax_tenths=10, acc_target=0.25, h_reset_each_cycle=0, bisect_iters=60,
                   seed=1, max_cycles=10000, nthreads=1)


def smc_run(spec, y, theta0, J, N, X=None, force_dates=(), design=None, record=False, burnin=0,
            pit=False, **kw):
    """Full adaptive run (Algorithm 2 with the Section 3.3 specifics).

    burnin=b > 0 (data tempering) also returns the log score log p(y_{b+1:T} |
    y_{1:b}) with its NSE; pit=True the probability integral transform of
    every observation (Section 4.1).

    record=True also returns the design of Algorithm 3 (end of each cycle, its
    iteration count and every iteration's proposal Cholesky factor);
    design=<that dict> replays it non-adaptively (Algorithm 3, step 2)."""
    o = dict(DEFAULT_RUN)
    o.update(kw)
    fd = np.ascontiguousarray(force_dates, dtype=np.int32)
    cap = 20000
    rec_L = np.zeros((cap, spec.d, spec.d)) if record else None
    if design is not None:
        dx = np.ascontiguousarray(design["x"], dtype=np.float64)
        dR = np.ascontiguousarray(design["R"], dtype=np.int32)
        dL = np.ascontiguousarray(design["L"], dtype=np.float64)
        rep = (1, len(dx), dx.ctypes.data_as(dp), dR.ctypes.data_as(ip), dL.ctypes.data_as(dp))
    else:
        rep = (0, 0, None, None, None)
    cfg = RunCfg(J, N, o["tempering"], o["mutation"], o["resid"], o["d1"], o["d2"],
                 o["stop_rule"], o["rbar"], o["kappa"], o["rmax"], o["e1"], o["e2"],
                 o["h0_tenths"], o["hmin_tenths"], o["hmax_tenths"], o["acc_target"],
                 o["h_reset_each_cycle"], fd.ctypes.data_as(ip) if len(fd) else None, len(fd),
                 o["bisect_iters"], o["seed"], o["max_cycles"], o["nthreads"], *rep,
                 rec_L.ctypes.data_as(dp) if record else None, cap if record else 0,
                 int(burnin), None)
    pit_arr = np.full(len(y), np.nan) if pit else None
    if pit:
        cfg.pit_out = pit_arr.ctypes.data_as(dp)
    P = J * N
    theta0 = _f64(theta0)
    assert theta0.shape == (P, spec.d)
    y = _f64(y)
    Xa = _f64(X) if X is not None else None
    theta = np.zeros((P, spec.d)); ll = np.zeros(P); lp = np.zeros(P)
    state = np.zeros((P, spec.nstate)); a = np.zeros(J)
    mc = o["max_cycles"]
    t_rec = np.zeros(mc, dtype=np.int32); phi_rec = np.zeros(mc)
    r_rec = np.zeros(mc, dtype=np.int32); rss_rec = np.zeros(mc)
    out = RunOut()
    _load().or_smc_run(C.byref(spec.c), _d(y), _d(Xa), len(y), C.byref(cfg), _d(theta0),
                       _d(theta), _d(ll), _d(lp), _d(state), _d(a),
                       t_rec.ctypes.data_as(ip), _d(phi_rec), r_rec.ctypes.data_as(ip),
                       _d(rss_rec), C.byref(out))
    L = out.cycles
    res_design = None
    if record:
        x = phi_rec[:L].copy() if o["tempering"] == 1 else t_rec[:L].astype(np.float64)
        res_design = dict(x=x, R=r_rec[:L].copy(), L=rec_L[:out.metropolis_steps].copy())
    return dict(status=out.status, cycles=L, metropolis_steps=out.metropolis_steps, design=res_design,
                evals=out.particle_obs_evals, log_ml=out.log_ml, log_ml_nse=out.log_ml_nse,
                log_ml_tilde=out.log_ml_tilde, h_final=out.h_final_tenths, theta=theta,
                log_score=out.log_score, log_score_nse=out.log_score_nse, pit=pit_arr,
                loglik=ll, logprior=lp, state=state, a=a, t=t_rec[:L].copy(),
                phi=phi_rec[:L].copy(), R=r_rec[:L].copy(), rss=rss_rec[:L].copy())
