"""ctypes binding of ``libsmc.so`` (C ABI in ``include/smc.h``).

Argument marshalling only: every step of the simulator runs in the library's
CUDA kernels.  Device buffers for the stateless entry points are torch CUDA
tensors (torch provides device memory and streams; it computes nothing here).
The library must be built (``python -m paper_1304_4334_gb300.build``); there is
no fallback path, so a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmc.so")
_lock = threading.Lock()
_lib = None

MAX_D, MAX_FORCE, MAX_N = 32, 64, 8192
OK, EINVAL, ENOMEM, ECUDA, EDEGENERATE, ENONFINITE, ETIMEOUT, EDONE = range(8)
EGARCH, LINREG = 0, 1
FP64, FP32 = 0, 1
DATA, POWER = 0, 1
RW, MALA, INDEP = 0, 1, 2
RESIDUAL, MULTINOMIAL, STRATIFIED, SYSTEMATIC = 0, 1, 2, 3
STOP_DET, STOP_RNE = 0, 1


class SMCError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"smc status {status}: {msg}")


class smc_model(C.Structure):
    _fields_ = [("model", C.c_int), ("K", C.c_int), ("I", C.c_int), ("gamma", C.c_int),
                ("eps0_zero", C.c_int), ("p", C.c_int), ("sigma", C.c_double),
                ("d_full", C.c_int), ("n_free", C.c_int), ("free_idx", C.c_int * MAX_D),
                ("theta_fixed", C.c_double * MAX_D), ("prior_mean", C.c_double * MAX_D),
                ("prior_sd", C.c_double * MAX_D), ("prior_lo", C.c_double * MAX_D)]

    @property
    def d(self):
        return self.n_free if self.n_free > 0 else self.d_full


class smc_config(C.Structure):
    _fields_ = [("J", C.c_int), ("N", C.c_int), ("precision", C.c_int), ("tempering", C.c_int),
                ("mutation", C.c_int), ("resampler", C.c_int), ("d1", C.c_double),
                ("d2", C.c_double), ("stop_rule", C.c_int), ("rbar", C.c_int),
                ("kappa", C.c_int), ("rmax", C.c_int), ("e1", C.c_double), ("e2", C.c_double),
                ("h0_tenths", C.c_int), ("hmin_tenths", C.c_int), ("hmax_tenths", C.c_int),
                ("acc_target", C.c_double), ("h_reset_each_cycle", C.c_int),
                ("n_force", C.c_int), ("force_dates", C.c_int * MAX_FORCE),
                ("search_passes", C.c_int), ("seed", C.c_uint64), ("burnin", C.c_int),
                ("pit", C.c_int)]


class smc_peak_rates(C.Structure):
    _fields_ = [("sms", C.c_int), ("ffma", C.c_double), ("ffma2", C.c_double), ("ex2", C.c_double),
                ("lg2", C.c_double), ("dfma", C.c_double), ("issue", C.c_double), ("sm_mhz", C.c_double),
                ("ffma_mix", C.c_double)]


class smc_cycle_info(C.Structure):
    _fields_ = [("cycle", C.c_int), ("t", C.c_int), ("phi", C.c_double), ("rss", C.c_double),
                ("R", C.c_int), ("h_tenths", C.c_int), ("acc_rate", C.c_double),
                ("evals", C.c_double), ("done", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


vp = C.c_void_p
dp = C.POINTER(C.c_double)


def _declare(L):
    P = C.POINTER
    L.smc_model_egarch.argtypes = [P(smc_model), C.c_int, C.c_int, C.c_int]
    L.smc_model_linreg.argtypes = [P(smc_model), C.c_int, C.c_double, dp, dp]
    L.smc_model_dim.argtypes = [P(smc_model)]
    L.smc_model_dim.restype = C.c_int
    L.smc_config_default.argtypes = [P(smc_config)]
    L.smc_config_default.restype = None
    L.smc_init.argtypes = [P(smc_model), P(smc_config), dp, dp, C.c_int, dp, C.c_int, vp, P(vp)]
    L.smc_cycle.argtypes = [vp, P(smc_cycle_info)]
    L.smc_run.argtypes = [vp, C.c_int, P(smc_cycle_info), P(C.c_int)]
    L.smc_log_ml.argtypes = [vp, dp, dp, dp]
    L.smc_log_score.argtypes = [vp, dp, dp]
    L.smc_wait_selftest.argtypes = [C.c_uint64, C.c_int, vp]
    L.smc_save.argtypes = [vp, C.c_char_p]
    L.smc_draw_prior.argtypes = [P(smc_model), C.c_uint64, C.c_int, vp, vp]
    L.smc_load.argtypes = [C.c_char_p, vp, P(vp)]
    L.smc_describe.argtypes = [vp, P(smc_model), P(smc_config), P(C.c_int)]
    L.smc_pit.argtypes = [vp, dp, C.c_int]
    L.smc_moments.argtypes = [vp, dp, P(C.c_int)]
    L.smc_group_estimators.argtypes = [vp, dp, dp]
    L.smc_peaks.argtypes = [P(smc_peak_rates), vp]
    L.smc_get_particles.argtypes = [vp, dp, dp, dp, dp]
    L.smc_launch_count.argtypes = []
    L.smc_launch_count.restype = C.c_uint64
    L.smc_profile.argtypes = [vp, C.c_int]
    L.smc_mutate_time.argtypes = [vp, dp, P(C.c_uint64), C.c_int]
    L.smc_reset.argtypes = [vp, dp, C.c_int, C.c_uint64]
    L.smc_run_totals.argtypes = [vp, P(C.c_int), P(C.c_int64), dp]
    L.smc_transfer_bytes.argtypes = [vp, P(C.c_uint64), P(C.c_uint64)]
    L.smc_free.argtypes = [vp]
    L.smc_free.restype = None
    L.smc_autotune.argtypes = [vp, C.c_int, P(C.c_int), P(C.c_int), dp]
    L.smc_set_launch_shape.argtypes = [vp, C.c_int, C.c_int]
    L.smc_design_record.argtypes = [vp, C.c_int]
    L.smc_design_size.argtypes = [vp, P(C.c_int), P(C.c_int)]
    L.smc_design_get.argtypes = [vp, dp, P(C.c_int), dp]
    L.smc_design_replay.argtypes = [vp, C.c_int, dp, P(C.c_int), dp]
    L.smc_batch_init.argtypes = [C.c_int, P(smc_model), P(smc_config), P(dp), P(C.c_int), P(dp), vp, P(vp)]
    L.smc_batch_autotune.argtypes = [vp, C.c_int, dp]
    L.smc_batch_cycle.argtypes = [vp, P(C.c_int)]
    L.smc_batch_run.argtypes = [vp, C.c_int, P(C.c_int)]
    L.smc_batch_reset.argtypes = [vp, P(dp), C.c_int, C.c_uint64]
    L.smc_batch_totals.argtypes = [vp, dp, P(C.c_int64), P(C.c_int)]
    L.smc_batch_member.argtypes = [vp, C.c_int]
    L.smc_batch_member.restype = vp
    L.smc_batch_tile.argtypes = [vp]
    L.smc_batch_tile.restype = C.c_int
    L.smc_batch_last_error.argtypes = [vp]
    L.smc_batch_last_error.restype = C.c_char_p
    L.smc_batch_free.argtypes = [vp]
    L.smc_batch_free.restype = None
    L.smc_last_error.argtypes = [vp]
    L.smc_last_error.restype = C.c_char_p
    L.smc_status_str.argtypes = [C.c_int]
    L.smc_status_str.restype = C.c_char_p
    L.smc_loglik.argtypes = [P(smc_model), C.c_int, vp, C.c_int, vp, C.c_int, vp, vp, vp, vp]
    L.smc_linreg_width.argtypes = [C.c_int]
    L.smc_linreg_width.restype = C.c_int
    L.smc_mutate_rw.argtypes = [P(smc_model), C.c_int, vp, C.c_int, vp, vp, vp, vp, C.c_int, vp,
                                C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, P(C.c_uint64), vp]
    L.smc_mutate_indep.argtypes = [P(smc_model), C.c_int, vp, C.c_int, vp, vp, vp, vp, C.c_int, vp, vp,
                                   C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, P(C.c_uint64), vp]
    L.smc_loglik_grad.argtypes = [P(smc_model), C.c_int, vp, C.c_int, vp, C.c_int, vp, vp, vp, vp]
    L.smc_mutate_mala.argtypes = [P(smc_model), C.c_int, vp, C.c_int, vp, vp, vp, vp, vp, C.c_int, vp,
                                  C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, P(C.c_uint64), vp]
    L.smc_cov_chol.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
    L.smc_power_search.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, vp]
    L.smc_resample.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, vp, vp]
    L.smc_resample_logw.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, vp, vp, vp]
    L.smc_group_moments.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, vp]
    L.smc_ml_from_groups.argtypes = [vp, C.c_int, dp, dp, vp]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1304_4334_gb300.build` (no fallback path exists)")
            _lib = C.CDLL(LIB_PATH)
            _declare(_lib)
    return _lib


def _check(st, ctx=None):
    if st != OK:
        L = lib()
        msg = L.smc_last_error(ctx).decode() if ctx else L.smc_status_str(st).decode()
        raise SMCError(st, msg)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a):
    return a.ctypes.data_as(dp) if a is not None else None


# ------------------------------------------------------------------- models
def model_egarch(K, I, gamma=True, eps0_zero=False, free_idx=None, theta_fixed=None):
    m = smc_model()
    _check(lib().smc_model_egarch(C.byref(m), K, I, int(bool(gamma))))
    m.eps0_zero = int(bool(eps0_zero))
    if free_idx is not None:
        _set_free(m, free_idx, theta_fixed)
    return m


def model_linreg(p, sigma, prior_mean, prior_sd):
    m = smc_model()
    pm, ps = _f64(prior_mean), _f64(prior_sd)
    _check(lib().smc_model_linreg(C.byref(m), p, sigma, _dptr(pm), _dptr(ps)))
    return m


def _set_free(m, free_idx, theta_fixed):
    """Keep only free_idx moving; the priors of the free parameters are taken
    from the full-model priors at those positions."""
    full_m = [m.prior_mean[i] for i in range(m.d_full)]
    full_s = [m.prior_sd[i] for i in range(m.d_full)]
    full_l = [m.prior_lo[i] for i in range(m.d_full)]
    m.n_free = len(free_idx)
    for k, i in enumerate(free_idx):
        m.free_idx[k] = int(i)
        m.prior_mean[k], m.prior_sd[k], m.prior_lo[k] = full_m[i], full_s[i], full_l[i]
    for i in range(m.d_full):
        m.theta_fixed[i] = float(theta_fixed[i])


def model_prior(m):
    d = m.d
    return (np.array(m.prior_mean[:d]), np.array(m.prior_sd[:d]), np.array(m.prior_lo[:d]))


def config_default(**kw):
    c = smc_config()
    lib().smc_config_default(C.byref(c))
    for k, v in kw.items():
        if k == "force_dates":
            c.n_force = len(v)
            for i, t in enumerate(v):
                c.force_dates[i] = int(t)
        else:
            setattr(c, k, v)
    return c


def peaks(stream=None):
    """Measured ALU pipe rates of the device (smc_peaks): lane operations per SM
    and clock for ffma, ffma2, ex2, lg2, dfma; warp instructions per SM and
    clock for issue; the SM clock (MHz) during the tests; the SM count."""
    r = smc_peak_rates()
    _check(lib().smc_peaks(C.byref(r), _stream(stream)))
    return {k: getattr(r, k) for k, _ in smc_peak_rates._fields_}


def launch_count():
    return int(lib().smc_launch_count())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


# ----------------------------------------------------------------- contexts
class Ctx:
    """A simulator run (wraps smc_ctx)."""

    def __init__(self, model, cfg, y, theta0, X=None, stream=None, theta0_on_device=False):
        self.model, self.cfg = model, cfg
        self.d = model.d
        self.P = cfg.J * cfg.N
        self._y = _f64(y)
        self.T = len(self._y)
        self._X = _f64(X) if X is not None else None
        h = C.c_void_p()
        if theta0_on_device:
            th_ptr = C.cast(C.c_void_p(theta0.data_ptr()), dp)
        else:
            self._th0 = _f64(theta0)
            assert self._th0.shape == (self.P, self.d), (self._th0.shape, self.P, self.d)
            th_ptr = _dptr(self._th0)
        st = lib().smc_init(C.byref(model), C.byref(cfg), _dptr(self._y), _dptr(self._X), len(self._y),
                            th_ptr, int(bool(theta0_on_device)), _stream(stream), C.byref(h))
        self.h = h
        if st != OK:
            msg = lib().smc_last_error(h).decode() if h else ""
            self.close()
            raise SMCError(st, msg)

    def cycle(self):
        info = smc_cycle_info()
        st = lib().smc_cycle(self.h, C.byref(info))
        if st == EDONE:
            return None
        _check(st, self.h)
        return info.as_dict()

    def run(self, max_cycles=0):
        info = smc_cycle_info()
        n = C.c_int()
        _check(lib().smc_run(self.h, max_cycles, C.byref(info), C.byref(n)), self.h)
        return n.value, info.as_dict()

    def reset(self, theta0, seed, theta0_on_device=False):
        if theta0_on_device:
            ptr = C.cast(C.c_void_p(theta0.data_ptr()), dp)
        else:
            self._th0 = _f64(theta0)
            ptr = _dptr(self._th0)
        _check(lib().smc_reset(self.h, ptr, int(bool(theta0_on_device)), seed), self.h)

    def totals(self):
        cyc, ms, ev = C.c_int(), C.c_int64(), C.c_double()
        _check(lib().smc_run_totals(self.h, C.byref(cyc), C.byref(ms), C.byref(ev)), self.h)
        return cyc.value, ms.value, ev.value

    def transfer_bytes(self):
        a, b = C.c_uint64(), C.c_uint64()
        _check(lib().smc_transfer_bytes(self.h, C.byref(a), C.byref(b)), self.h)
        return a.value, b.value

    def log_ml(self):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        _check(lib().smc_log_ml(self.h, C.byref(a), C.byref(b), C.byref(c)), self.h)
        return a.value, b.value, c.value

    def group_estimators(self):
        """(a_j, log wbar_j(l-1) of the last cycle) per group (smc_group_estimators)."""
        a = np.zeros(self.cfg.J)
        lw = np.zeros(self.cfg.J)
        _check(lib().smc_group_estimators(self.h, _dptr(a), _dptr(lw)), self.h)
        return a, lw

    def log_score(self):
        """(log p(y_{b+1:T} | y_1:b), NSE) for the configured burn-in b."""
        a, b = C.c_double(), C.c_double()
        _check(lib().smc_log_score(self.h, C.byref(a), C.byref(b)), self.h)
        return a.value, b.value

    def pit(self):
        """Probability integral transform of every observation (NaN until reached)."""
        out = np.zeros(self.T)
        _check(lib().smc_pit(self.h, _dptr(out), self.T), self.h)
        return out

    def moments(self):
        out = np.zeros((self.d + 3, 4))
        nf = C.c_int()
        _check(lib().smc_moments(self.h, _dptr(out), C.byref(nf)), self.h)
        return out[:nf.value]

    def particles(self):
        th = np.zeros((self.P, self.d))
        ll = np.zeros(self.P)
        lp = np.zeros(self.P)
        ns = self.model.K + 1 if self.model.model == EGARCH else 0
        st = np.zeros((self.P, max(ns, 1)))
        _check(lib().smc_get_particles(self.h, _dptr(th), _dptr(ll), _dptr(lp),
                                       _dptr(st) if ns else None), self.h)
        return th, ll, lp, st[:, :ns]

    def autotune(self, iters=2):
        """Pick the mutation kernel's launch shape by timing (smc_autotune)."""
        ppt, thr, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lib().smc_autotune(self.h, iters, C.byref(ppt), C.byref(thr), C.byref(ms)), self.h)
        return ppt.value, thr.value, ms.value

    def set_launch_shape(self, ppt, threads):
        _check(lib().smc_set_launch_shape(self.h, ppt, threads), self.h)

    # Algorithm 3 (hybrid)
    def record_design(self, max_iterations=4096):
        _check(lib().smc_design_record(self.h, max_iterations), self.h)

    def design(self):
        nc, ni = C.c_int(), C.c_int()
        _check(lib().smc_design_size(self.h, C.byref(nc), C.byref(ni)), self.h)
        x = np.zeros(nc.value)
        R = np.zeros(nc.value, dtype=np.int32)
        L = np.zeros((ni.value, self.d, self.d))
        _check(lib().smc_design_get(self.h, _dptr(x), R.ctypes.data_as(C.POINTER(C.c_int)),
                                    _dptr(L) if ni.value else None), self.h)
        return {"x": x, "R": R, "L": L}

    def replay_design(self, design):
        x = _f64(design["x"])
        R = np.ascontiguousarray(design["R"], dtype=np.int32)
        L = _f64(design["L"])
        self._design = (x, R, L)
        _check(lib().smc_design_replay(self.h, len(x), _dptr(x), R.ctypes.data_as(C.POINTER(C.c_int)),
                                       _dptr(L)), self.h)

    def profile(self, enable=True):
        """True or 1: time every mutation launch; 2: the first of each M phase."""
        _check(lib().smc_profile(self.h, int(enable)), self.h)

    def mutate_time(self, reset=False):
        ms = C.c_double()
        n = C.c_uint64()
        _check(lib().smc_mutate_time(self.h, C.byref(ms), C.byref(n), int(reset)), self.h)
        return ms.value, n.value

    def save(self, path):
        """Checkpoint the run between cycles (smc_save)."""
        _check(lib().smc_save(self.h, str(path).encode()), self.h)

    @classmethod
    def load(cls, path, stream=None):
        """A context resumed from a checkpoint file (smc_load)."""
        h = C.c_void_p()
        st = lib().smc_load(str(path).encode(), _stream(stream), C.byref(h))
        if st != OK:
            raise SMCError(st, "smc_load failed")
        self = cls.__new__(cls)
        self.h = h
        m, c, T = smc_model(), smc_config(), C.c_int()
        _check(lib().smc_describe(h, C.byref(m), C.byref(c), C.byref(T)), h)
        self.model, self.cfg = m, c
        self.d = m.n_free if m.n_free > 0 else m.d_full
        self.P = c.J * c.N
        self.T = T.value
        return self

    def close(self):
        if getattr(self, "h", None):
            lib().smc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _MemberView(Ctx):
    """A batch member's context (owned by the batch: close() does nothing)."""

    def __init__(self, handle, model, cfg):
        self.h = handle
        self.model, self.cfg = model, cfg
        self.d = model.d
        self.P = cfg.J * cfg.N

    def close(self):
        self.h = None


class Batch:
    """Many runs advanced together (wraps smc_batch)."""

    def __init__(self, models, cfgs, ys, theta0s, stream=None):
        n = len(models)
        self.models, self.cfgs = list(models), list(cfgs)
        self._ys = [_f64(y) for y in ys]
        self._th = [_f64(t) for t in theta0s]
        M = (smc_model * n)(*self.models)
        Cf = (smc_config * n)(*self.cfgs)
        Y = (dp * n)(*[_dptr(y) for y in self._ys])
        Ts = (C.c_int * n)(*[len(y) for y in self._ys])
        TH = (dp * n)(*[_dptr(t) for t in self._th])
        self._keep = (M, Cf, Y, Ts, TH)
        h = C.c_void_p()
        st = lib().smc_batch_init(n, M, Cf, Y, Ts, TH, _stream(stream), C.byref(h))
        self.h = h
        self.n = n
        if st != OK:
            msg = lib().smc_batch_last_error(h).decode() if h else ""
            self.close()
            raise SMCError(st, msg)

    def _chk(self, st):
        if st != OK:
            raise SMCError(st, lib().smc_batch_last_error(self.h).decode())

    def autotune(self, iters=2):
        ms = C.c_double()
        self._chk(lib().smc_batch_autotune(self.h, iters, C.byref(ms)))
        return ms.value

    @property
    def tile(self):
        return lib().smc_batch_tile(self.h)

    def cycle(self):
        n = C.c_int()
        st = lib().smc_batch_cycle(self.h, C.byref(n))
        if st == EDONE:
            return None
        self._chk(st)
        return n.value

    def run(self, max_cycles=0):
        n = C.c_int()
        self._chk(lib().smc_batch_run(self.h, max_cycles, C.byref(n)))
        return n.value

    def reset(self, theta0s, seed, on_device=True):
        if on_device:
            ptrs = [C.cast(C.c_void_p(t.data_ptr()), dp) for t in theta0s]
        else:
            self._th = [_f64(t) for t in theta0s]
            ptrs = [_dptr(t) for t in self._th]
        arr = (dp * self.n)(*ptrs)
        self._chk(lib().smc_batch_reset(self.h, arr, int(bool(on_device)), seed))

    def totals(self):
        e, ms, cy = C.c_double(), C.c_int64(), C.c_int()
        self._chk(lib().smc_batch_totals(self.h, C.byref(e), C.byref(ms), C.byref(cy)))
        return e.value, ms.value, cy.value

    def member(self, i):
        return _MemberView(lib().smc_batch_member(self.h, i), self.models[i], self.cfgs[i])

    def close(self):
        if getattr(self, "h", None):
            lib().smc_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def init(model, cfg, y, theta0, X=None, stream=None, theta0_on_device=False):
    return Ctx(model, cfg, y, theta0, X=X, stream=stream, theta0_on_device=theta0_on_device)


def load(path, stream=None):
    return Ctx.load(path, stream=stream)


def draw_prior(model, seed, P, stream=None):
    """Table 1 prior draws on the device: a float64 cuda tensor [d, P]."""
    import torch
    th = torch.empty((model.d, P), dtype=torch.float64, device="cuda")
    _check(lib().smc_draw_prior(C.byref(model), seed, P, _ptr(th), _stream(stream)))
    return th


# ------------------------------------------------ stateless (torch device buffers)
def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def linreg_width(p):
    return lib().smc_linreg_width(p)


def loglik(model, precision, obs, theta, ll, lp=None, state=None, stream=None):
    """obs: device tensor (float32 [T] for FP32 EGARCH, float64 otherwise);
    theta: float64 [d, P]; outputs float64 tensors."""
    T = obs.shape[0]
    P = theta.shape[1]
    _check(lib().smc_loglik(C.byref(model), precision, _ptr(obs), T, _ptr(theta), P, _ptr(ll),
                            _ptr(lp), _ptr(state), _stream(stream)))


def mutate_rw(model, precision, obs, theta, ll, lp, state, L, phi, seed, cycle, it, stream=None):
    T = obs.shape[0]
    P = theta.shape[1]
    acc = C.c_uint64()
    _check(lib().smc_mutate_rw(C.byref(model), precision, _ptr(obs), T, _ptr(theta), _ptr(ll),
                               _ptr(lp), _ptr(state), P, _ptr(L), float(phi), seed, cycle, it,
                               C.byref(acc), _stream(stream)))
    return acc.value


def wait_selftest(limit_ns, complete, stream=None):
    """Status of the bounded-wait self-test (ETIMEOUT when the wait ran out)."""
    return lib().smc_wait_selftest(int(limit_ns), int(bool(complete)), _stream(stream))


def mutate_indep(model, precision, obs, theta, ll, lp, state, mean, L, phi, seed, cycle, it, stream=None):
    """One independent Gaussian Metropolis iteration, proposal N(mean, L L')."""
    T = obs.shape[0]
    P = theta.shape[1]
    acc = C.c_uint64()
    _check(lib().smc_mutate_indep(C.byref(model), precision, _ptr(obs), T, _ptr(theta), _ptr(ll),
                                  _ptr(lp), _ptr(state), P, _ptr(mean), _ptr(L), float(phi), seed, cycle,
                                  it, C.byref(acc), _stream(stream)))
    return acc.value


def loglik_grad(model, precision, obs, theta, ll, grad, state=None, stream=None):
    """Log likelihood and its theta-gradient (adjoint kernel); grad float64 [d, P]."""
    T = obs.shape[0]
    P = theta.shape[1]
    _check(lib().smc_loglik_grad(C.byref(model), precision, _ptr(obs), T, _ptr(theta), P, _ptr(ll),
                                 _ptr(grad), _ptr(state), _stream(stream)))


def mutate_mala(model, precision, obs, theta, ll, lp, grad, state, L, phi, seed, cycle, it, stream=None):
    T = obs.shape[0]
    P = theta.shape[1]
    acc = C.c_uint64()
    _check(lib().smc_mutate_mala(C.byref(model), precision, _ptr(obs), T, _ptr(theta), _ptr(ll),
                                 _ptr(lp), _ptr(grad), _ptr(state), P, _ptr(L), float(phi), seed, cycle,
                                 it, C.byref(acc), _stream(stream)))
    return acc.value


def cov_chol(theta, h_tenths, mean=None, cov=None, L=None, stream=None):
    d, P = theta.shape
    _check(lib().smc_cov_chol(_ptr(theta), d, P, h_tenths, _ptr(mean), _ptr(cov), _ptr(L),
                              _stream(stream)))


def power_search(ll, phi, d1=0.5, passes=6, stream=None):
    dphi, rss = C.c_double(), C.c_double()
    _check(lib().smc_power_search(_ptr(ll), ll.shape[0], float(phi), float(d1), passes,
                                  C.byref(dphi), C.byref(rss), _stream(stream)))
    return dphi.value, rss.value


def resample(w, J, N, idx, resampler=RESIDUAL, seed=0, cycle=0, stream=None):
    _check(lib().smc_resample(_ptr(w), J, N, resampler, seed, cycle, _ptr(idx), _stream(stream)))


def resample_logw(logw, J, N, idx, resampler=RESIDUAL, seed=0, cycle=0, stream=None):
    """S phase from log weights; returns log wbar_j of each group (host [J])."""
    lwbar = np.zeros(J)
    _check(lib().smc_resample_logw(_ptr(logw), J, N, resampler, seed, cycle, _ptr(idx), _dptr(lwbar),
                                   _stream(stream)))
    return lwbar


def group_moments(g, J, N, stream=None):
    nf = g.shape[0]
    out = np.zeros((nf, 4))
    _check(lib().smc_group_moments(_ptr(g), nf, J, N, _dptr(out), _stream(stream)))
    return out


def ml_from_groups(a, stream=None):
    x, s = C.c_double(), C.c_double()
    _check(lib().smc_ml_from_groups(_ptr(a), a.shape[0], C.byref(x), C.byref(s), _stream(stream)))
    return x.value, s.value
