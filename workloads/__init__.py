"""Seeded synthetic inputs for batched OMP (dictionaries and planted sparse signals).

This package is shared by the FP64 oracle, the tests and the benchmark. It holds only the input
model y = A x + noise of the problem statement (paper Sec. 1); none of OMP's own arithmetic.
"""
from .gen import (  # noqa: F401
    CONFIGS,
    Workload,
    get_config,
    dictionary,
    planted,
    signals,
    synthesize,
    training_batch,
)
