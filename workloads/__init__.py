"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds only input generation (counter-based random numbers and
the shape lists of the workloads).  It contains none of the GEMM or
selection arithmetic, so both the CPU oracle and the GPU path may import it
without sharing any of the method's code.
"""

from .rng import (  # noqa: F401
    splitmix64,
    uniform_pm1,
    small_ints,
    normal,
    log_uniform_signed,
    matrix,
    rank1_operands,
    wide_int_operands,
)
from .shapes import (  # noqa: F401
    SWEEP_SIZES,
    sweep_shapes,
    parity_split,
    random_split,
    split_precision_shapes,
    grouped_problems,
)
