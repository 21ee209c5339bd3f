"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package draws matrices and right-hand sides only.  It holds none of the
solver's arithmetic, so both the CUDA path and the CPU oracle can consume its
output without sharing any code with each other.
"""

from .gen import (  # noqa: F401
    Workload,
    RhsSet,
    dominant_blocks,
    uniform_rhs,
    poisson_system,
    poisson_manufactured,
    pml_sigma,
    acoustic_system,
    acoustic_rhs,
    batched_sets,
    config0,
    config1,
    config2,
    config3,
    config4,
)
