"""smc_cov_chol_noalloc through the C ABI: the covariance + Cholesky entry point
for callers that cannot allocate device memory while they run.  Its scratch is
a fixed array inside the library; its results must match the allocating
smc_cov_chol on three calls in a row whose shapes shrink and then grow (so
stale scratch contents of an earlier call would show).  Both entry points split
the particles over the same blocks, so on a device with up to 256 SMs the
results are identical; the test also checks them against numpy."""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import host, soa, torch_cuda

pytestmark = pytest.mark.gpu


def test_cov_chol_noalloc_matches_allocating_entry_point():
    torch = torch_cuda()
    from paper_1304_4334_gb300 import build
    build.build()
    from paper_1304_4334_gb300 import smc
    lib = smc.lib()
    fn = lib.smc_cov_chol_noalloc
    fn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    same_partition = torch.cuda.get_device_properties(0).multi_processor_count <= 256
    for d, P, h, seed in [(14, 65536 + 37, 7, 1), (5, 3001, 4, 2), (3, 97, 10, 3), (20, 400000 + 5, 6, 4)]:
        rng = np.random.default_rng(seed)
        th = rng.normal(size=(P, d)) @ (0.1 * rng.normal(size=(d, d))) + rng.normal(0, 3, d)
        tg = soa(th)
        outs = []
        for which in ("alloc", "noalloc"):
            mean = torch.full((d,), np.nan, dtype=torch.float64, device="cuda")
            cov = torch.full((d, d), np.nan, dtype=torch.float64, device="cuda")
            L = torch.full((d, d), np.nan, dtype=torch.float64, device="cuda")
            if which == "alloc":
                smc.cov_chol(tg, h, mean, cov, L)
            else:
                st = fn(C.c_void_p(tg.data_ptr()), d, P, h, C.c_void_p(mean.data_ptr()),
                        C.c_void_p(cov.data_ptr()), C.c_void_p(L.data_ptr()), stream)
                assert st == smc.OK
            torch.cuda.synchronize()
            outs.append((host(mean), host(cov), host(L)))
        (m0, c0, l0), (m1, c1, l1) = outs
        if same_partition:
            np.testing.assert_array_equal(m1, m0)
            np.testing.assert_array_equal(c1, c0)
            np.testing.assert_array_equal(l1, l0)
        sd = np.sqrt(np.diag(c0))
        np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-6 * sd.max())
        np.testing.assert_allclose(c1, c0, rtol=1e-5, atol=1e-6 * np.abs(c0).max())
        np.testing.assert_allclose(l1, l0, rtol=1e-4, atol=1e-5 * np.abs(l0).max())
        np.testing.assert_allclose(c1, np.cov(th.T), rtol=1e-5, atol=1e-6 * np.abs(c0).max())
    # sizes beyond the stated maximum are rejected before any device work
    assert fn(C.c_void_p(tg.data_ptr()), smc.MAX_D + 1, 100, 5, None, None, None, stream) == smc.EINVAL
    assert fn(C.c_void_p(tg.data_ptr()), 3, 1, 5, None, None, None, stream) == smc.EINVAL
