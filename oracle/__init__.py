"""CPU FP64 oracle for the staggered Dslash / even-odd CG path (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg import this package.
"""
from . import staggered  # noqa: F401
