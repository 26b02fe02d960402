"""SplitMix64 streams for coefficients and right-hand sides.

SplitMix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then the output
is the state mixed by two xor-shift-multiply rounds.  A 53-bit mantissa of each
output gives u in [0, 1).  Both the CUDA path and the oracle receive arrays made
here; neither draws random numbers itself.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of SplitMix64(seed) as float64 in [0, 1)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def rhs_vector(seed: int, n: int, nrhs: int = 1) -> np.ndarray:
    """Right-hand side(s), i.i.d. uniform in [-1, 1); column j uses seed + 1000 j.

    Returned row-major [n] for nrhs == 1, else [n][nrhs] (right-hand sides contiguous).
    """
    if nrhs == 1:
        return 2.0 * splitmix64_uniform(seed, n) - 1.0
    cols = [2.0 * splitmix64_uniform(seed + 1000 * j, n) - 1.0 for j in range(nrhs)]
    return np.ascontiguousarray(np.stack(cols, axis=1))


def block_coefficients(n: int, block: int, lo_exp: float, hi_exp: float, seed: int) -> np.ndarray:
    """Per-tetrahedron coefficient, constant on block^3 groups of cubes, 10^U(lo, hi).

    Blocks are drawn in block-major order (bx, by, bz); tet t of cube (a, b, c) is
    t = 6 ((a n + b) n + c) + permutation, matching the mesh generator.
    """
    nb = (n + block - 1) // block
    u = splitmix64_uniform(seed, nb ** 3)
    val = 10.0 ** (lo_exp + (hi_exp - lo_exp) * u)
    a, b, c = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    blk = ((a // block) * nb + (b // block)) * nb + (c // block)
    per_cube = val[blk.reshape(-1)]
    return np.repeat(per_cube, 6)


def workload_coefficients(n: int, contrast_blocks: bool, seed: int):
    """(beta, alpha) per tet: beta multiplies (Du, Dv), alpha multiplies (u, v).

    contrast_blocks: beta log-uniform in [1e-3, 1e3] per 8^3 block of cubes, else 1;
    alpha = 1 everywhere.
    """
    alpha = np.ones(6 * n ** 3)
    if contrast_blocks:
        beta = block_coefficients(n, 8, -3.0, 3.0, seed)
    else:
        beta = np.ones(6 * n ** 3)
    return beta, alpha
