"""CPU FP64 oracle of the AMGe solve phase -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline / reference
legs may import this package.  The CUDA solve library never calls it, links it or
falls back to it.  It shares no code with the CUDA path: both read the same
generated hierarchy arrays (paper_2107_05613_gb300.inputs) and nothing else.
"""
from .amge_oracle import (
    AuxSpaceCoarseSolver,
    OracleHierarchy,
    SymmetricGaussSeidel,
    coarse_interpolation,
    colour_order,
    greedy_colours,
    l1_row_sums,
    pcg,
)

__all__ = ["AuxSpaceCoarseSolver", "OracleHierarchy", "SymmetricGaussSeidel", "coarse_interpolation", "colour_order",
           "greedy_colours", "l1_row_sums", "pcg"]
