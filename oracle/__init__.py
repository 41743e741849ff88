"""Plain FP64 CPU oracle for the sequential posterior simulator.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of ``bench.py``.  The product path never imports it.
"""
from .oracle import *  # noqa: F401,F403
