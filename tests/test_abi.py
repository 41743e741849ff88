"""Host-side checks of the C ABI library (no GPU needed): it builds, loads,
exports every function include/smc.h declares, and its host-only helpers
agree with the paper's tables."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_1304_4334_gb300 import build as B
from tests.golden_io import defaults, table1_vector

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def smc():
    B.build()
    from paper_1304_4334_gb300 import smc as S
    S.lib()
    return S


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(smc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["smc_init", "smc_cycle", "smc_log_ml", "smc_moments", "smc_free", "smc_loglik",
                 "smc_mutate_rw", "smc_cov_chol", "smc_power_search", "smc_resample"]:
        assert must in names


def test_library_exports_every_declared_symbol(smc):
    L = smc.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("K,I,gamma", [(1, 1, False), (2, 2, True), (3, 4, True), (4, 3, False)])
def test_table1_priors_in_library(smc, K, I, gamma):
    m = smc.model_egarch(K, I, gamma)
    mean, sd, lo = smc.model_prior(m)
    wm, ws, wl = table1_vector(K, I, gamma)
    np.testing.assert_allclose(mean, wm, atol=1e-15)
    np.testing.assert_allclose(sd, ws, atol=1e-15)
    assert np.array_equal(np.isinf(lo), np.isinf(wl)) and np.all(lo[~np.isinf(lo)] == np.array(wl)[~np.isinf(wl)])
    assert smc.lib().smc_model_dim(C.byref(m)) == len(wm)


def test_config_defaults_match_section_3_3(smc):
    c = smc.config_default()
    d = defaults()
    assert (c.d1, c.d2, c.rbar, c.kappa) == (d["D1"], d["D2"], d["Rbar"], d["kappa"])
    assert (c.e1, c.e2, c.rmax) == (d["E1"], d["E2"], d["Rmax"])
    assert c.h0_tenths / 10 == d["h0"] and c.hmin_tenths / 10 == d["h_min"]
    assert c.hmax_tenths / 10 == d["h_max"] and c.acc_target == d["acc_target"]
    assert c.resampler == smc.RESIDUAL and c.mutation == smc.RW


def test_init_rejects_bad_arguments_before_touching_the_device(smc):
    m = smc.model_egarch(1, 1, False)
    y = np.zeros(10)
    th = np.zeros((8, m.d))
    for kw in [dict(J=1, N=8), dict(J=2, N=smc.MAX_N + 1), dict(J=2, N=4, d1=1.5),
               dict(J=2, N=4, h0_tenths=11), dict(J=2, N=4, precision=7)]:
        c = smc.config_default(**kw)
        with pytest.raises(smc.SMCError) as e:
            smc.init(m, c, y, np.zeros((c.J * c.N, m.d)), stream=0)
        assert e.value.status == smc.EINVAL
    c = smc.config_default(J=2, N=4)
    y_bad = y.copy()
    y_bad[3] = math.nan
    with pytest.raises(smc.SMCError) as e:
        smc.init(m, c, y_bad, th, stream=0)
    assert e.value.status == smc.ENONFINITE


def test_linreg_width(smc):
    assert [smc.linreg_width(p) for p in range(1, 8)] == [2, 4, 4, 8, 8, 8, 8]
