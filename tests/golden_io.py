"""Readers for the small text fixtures under tests/golden/ (each cites its source)."""
import math
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_FUNCS = {"log": math.log, "atanh": math.atanh, "inf": math.inf}


def _num(tok):
    tok = tok.strip()
    if tok in ("-inf", "inf"):
        return float(tok)
    return float(eval(tok, {"__builtins__": {}}, _FUNCS))


def table1():
    """name -> (mean, sd, lo) from Table 1."""
    out = {}
    with open(os.path.join(GOLDEN, "table1_priors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, mean, sd, lo, _ = line.split()
            out[name] = (_num(mean), _num(sd), _num(lo))
    return out


def table1_vector(K, I, gamma=True):
    t = table1()
    rows = [t["theta1"], t["theta2"]] + [t["theta3k"]] * K + [t["theta4k"]] * K
    if gamma:
        rows += [t["theta5k"]] * K
    if I >= 2:
        rows += [t["theta6i"]] * I + [t["theta7i"]] * I + [t["theta8i"]] * I
    return tuple(list(x) for x in zip(*rows))


def defaults():
    out = {}
    with open(os.path.join(GOLDEN, "section3_defaults.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out
