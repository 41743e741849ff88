"""Pins for the oracle's Philox4x64-10 and its normal/uniform draws.

Philox is pinned to numpy.random.Philox, an independent implementation of the
same published generator (Salmon et al., SC'11).  numpy increments its counter
before producing a block, so numpy at counter c-1 yields Philox(c)."""
import numpy as np
import pytest
from scipy import stats

import oracle as O

CASES = [
    ((1, 0, 0, 0), (0, 0)),
    ((7, 3, 2, (1 << 32) | 5), (12345, 0)),
    ((2 ** 63, 2 ** 40 + 9, 17, 3 << 32), (0xDEADBEEFCAFEBABE, 0)),
    ((99, 0, 1, 0), (2 ** 64 - 1, 7)),
]


@pytest.mark.parametrize("ctr,key", CASES)
def test_philox_matches_numpy(ctr, key):
    prev = list(ctr)
    prev[0] -= 1           # every case has ctr[0] >= 1, so no borrow
    bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    want = bg.random_raw(4)
    got = O.philox4x64(ctr, key)
    assert np.array_equal(got, want)


def test_philox_counter_sensitivity():
    a = O.philox4x64((5, 0, 0, 0), (1, 0))
    for i in range(4):
        c = [5, 0, 0, 0]
        c[i] ^= 1
        b = O.philox4x64(tuple(c), (1, 0))
        bits = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
        assert 80 < bits < 176      # avalanche: about half of 256 bits flip


def test_normals_are_standard():
    z = np.concatenate([O.philox_normals(7, p, 0, 1, 14) for p in range(3000)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_normals_depend_on_every_counter_field():
    base = O.philox_normals(1, 3, 4, 5, 6)
    for args in [(2, 3, 4, 5), (1, 4, 4, 5), (1, 3, 5, 5), (1, 3, 4, 6)]:
        assert not np.allclose(O.philox_normals(*args, 6), base)


def test_log_uniform_is_uniform():
    u = np.exp([O.philox_log_uniform(3, p, 2, 9) for p in range(5000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert u.min() > 0.0 and u.max() < 1.0
