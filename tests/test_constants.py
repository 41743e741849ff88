"""Every long decimal constant written into the CUDA sources, checked against
its mathematical definition (CPU only).

The FP32 recursion runs in scaled units (base-2 logarithms, shocks scaled by
s = (log2(e)/2)^1/2), so it carries constants such as ln s and log2 s that
enter every observation's log density; a digit typed wrong there biases the
log likelihood by the same amount at every observation, which a relative
tolerance of 1e-4 on one evaluation does not see.  Each literal with six or
more fractional digits must appear in the table below with its definition,
and must equal it to double precision.
"""
import math
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1304_4334_gb300", "csrc")

S = math.sqrt(math.log2(math.e) / 2.0)
DEFINITIONS = {
    "1.83787706640934548356": math.log(2.0 * math.pi),       # ln(2 pi)
    "0.79788456080286535588": math.sqrt(2.0 / math.pi),      # (2/pi)^1/2 of (EGARCH_mod1)
    "0.69314718055994530942": math.log(2.0),
    "1.44269504088896340736": 1.0 / math.log(2.0),           # log2(e)
    "0.84932180028801904272": S,
    "0.23561681352755119288": -math.log2(S),                 # written with its minus sign
    "0.16331712998914049120": -math.log(S),
    "0.70710678118654752440": math.sqrt(0.5),
    "2.3283064365386963e-10": 2.0 ** -32,
}


def _literals():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith((".cu", ".cuh", ".h")):
            continue
        for i, line in enumerate(open(os.path.join(CSRC, f)), start=1):
            for m in re.finditer(r"(?<![\w.])(\d+\.\d{6,}(?:e-?\d+)?)f?", line):
                out.append((f, i, m.group(1)))
    return out


def test_every_long_constant_is_defined_and_exact():
    found = _literals()
    assert len(found) >= 8
    for f, i, lit in found:
        assert lit in DEFINITIONS, f"{f}:{i}: literal {lit} has no definition in this test"
        want = DEFINITIONS[lit]
        assert abs(float(lit) - want) <= 5e-16 * abs(want), (f, i, lit, want)   # a few ulp


def test_scaled_unit_identities():
    """The relations the FP32 recursion relies on: log2(e)/2 = s^2, and ln s,
    log2 s consistent with each other through ln 2."""
    s = float("0.84932180028801904272")
    assert abs(s * s - math.log2(math.e) / 2.0) < 1e-16
    l2 = -float("0.23561681352755119288")
    ln = -float("0.16331712998914049120")
    assert abs(ln - l2 * math.log(2.0)) < 1e-16
    assert abs(2.0 ** l2 - s) < 1e-16


def test_fixed_point_exponential_table():
    """The S phase's fixed-point exponential: round(ln 2 2^64),
    round(256/ln 2 2^50) and the 256 powers round(2^(63 - j/256)), checked
    with exact decimal arithmetic, plus the identities a wrong entry breaks:
    the table is strictly decreasing, and T[j] T[256 - j] = 2^125 within the
    rounding of two entries."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    src = open(os.path.join(CSRC, "exp2_table.h")).read()
    ln2 = Decimal(2).ln()
    l64 = int(re.search(r"kLn2Q64 = (\d+)ull", src).group(1))
    r50 = int(re.search(r"kInvLn2x256Q50 = (\d+)ull", src).group(1))
    assert l64 == int((ln2 * 2 ** 64).to_integral_value())
    assert r50 == int((Decimal(256) / ln2 * 2 ** 50).to_integral_value())
    body = src[src.index("g_exp2_neg256"):]
    tab = [int(t) for t in re.findall(r"(\d+)ull", body)]
    assert len(tab) == 256 and tab[0] == 2 ** 63
    for j, t in enumerate(tab):
        exact = Decimal(2) ** (Decimal(63) - Decimal(j) / 256)
        assert abs(Decimal(t) - exact) <= Decimal("0.5"), j
    assert all(a > b for a, b in zip(tab, tab[1:]))
    for j in range(1, 256):
        prod = Decimal(tab[j]) * Decimal(tab[256 - j]) if j != 128 else Decimal(tab[128]) ** 2
        assert abs(prod / Decimal(2) ** 125 - 1) < Decimal(2) ** -61, j
