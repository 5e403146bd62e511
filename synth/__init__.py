"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the benchmark.

This package holds only case parameters and random draws (a splitmix64 stream); it holds
none of the method's arithmetic.  Each implementation (the CPU oracle and the CUDA library)
turns these parameters into states with its own equations of state.
"""
from .cases import (  # noqa: F401
    CASE_KEYS,
    splitmix64_uniform,
    nozzle_case,
    plume_case,
    plume_case_mixed_precision,
    batch_cases,
    mixing_layer_case,
    freezing_case,
    closed_box_case,
    shock_tube_case,
)
