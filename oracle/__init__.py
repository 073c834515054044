"""Plain FP64 CPU oracle for the Fast chi-squared periodogram (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package.  The CUDA library neither imports nor links it.
"""
from .oracle import *  # noqa: F401,F403
