"""Seeded synthetic inputs shared by the CUDA solve path and the CPU oracle.

Nothing here applies the solve-phase method (no smoothing, no V-cycle, no Krylov
step): it generates the problem data both sides consume -- the AMGe de Rham
hierarchy built once on the host in FP64 (Sections 2-3 of the paper, as input
data), per-element coefficients, and right-hand sides from SplitMix64.
"""
from .rng import splitmix64_uniform, block_coefficients, rhs_vector, workload_coefficients
from .hierarchy import build_hierarchy, hierarchy_to_blob, Hierarchy, CSR

__all__ = [
    "splitmix64_uniform",
    "block_coefficients",
    "rhs_vector",
    "workload_coefficients",
    "build_hierarchy",
    "Hierarchy",
    "CSR",
    "hierarchy_to_blob",
]
