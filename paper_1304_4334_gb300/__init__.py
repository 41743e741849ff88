"""GB300-native sequential posterior simulator (Durham & Geweke, 2013).

The compute path is the C-ABI library ``libsmc.so`` (hand-written sm_103a CUDA,
built from ``csrc/``); :mod:`paper_1304_4334_gb300.smc` is its ctypes binding.
Importing the package loads nothing; the binding loads the library on first use
and raises if it has not been built.
"""
__all__ = ["smc", "inputs"]
