"""Plain FP64 CPU oracle for Piacsek-Williams advection (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package. The GPU library never imports it, and it imports nothing
from the GPU library.
"""
from .oracle import (  # noqa: F401
    build_oracle,
    coeffs,
    advect,
    advect_adjoint,
    monomial_scale,
    energy_weights,
    energy_budget,
    flops_per_column,
)
