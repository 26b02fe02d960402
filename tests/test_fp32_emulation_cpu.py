"""Why the FP32 V-cycle computes some residuals on the FP64 operator (CPU only).

With the derivative coefficient jumping by 1e6 between blocks, the large-coefficient
part of A_l annihilates gradients (H(curl)) and curls (H(div)) exactly, so for an
iterate x that carries a correction through G or P most of A_l x cancels.  An FP32
residual b - A_l x then carries a rounding error of order eps_32 |A_l| |x| in its
gradient (curl) part, which the aux sweep and the coarse solve divide by mass-only
diagonals.  The CPU emulation (tests/fp32_emulation.py) of the CUDA V-cycle's steps
shows it: on the 32^3 contrast workloads an all-FP32 cycle is several percent off in
the energy norm (on 64^3 the FP32 PCG stagnates near relres 0.17 and 0.05), while
computing the residuals of corrected iterates with FP64 values and sums brings the
cycle to ~5e-5.  The emulation itself is pinned first: in FP64 it must reproduce the
oracle's V-cycle (its A G update and residue drop are exact rewrites up to rounding).
"""
import numpy as np
import pytest

from conftest import hierarchy, oracle_hierarchy
import fp32_emulation
from fp32_emulation import EmulatedVcycle, energy_error, policy_df, policy_fp32, policy_fp64, policy_wide, resid_df
from paper_2107_05613_gb300.inputs import rhs_vector


@pytest.mark.parametrize("form,n,L", [("hcurl", 8, 2), ("hdiv", 8, 3), ("hcurl", 16, 2)])
def test_emulation_in_fp64_is_the_oracle_vcycle(form, n, L):
    hh = hierarchy(form, n, L, True)
    o = oracle_hierarchy(form, n, L, True)
    r = rhs_vector(5, hh.A[0].shape[0])
    ref = o.apply(r)
    z = EmulatedVcycle(hh, policy_fp64, vec=np.float64).apply(r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_fp32_residuals_of_corrected_iterates_need_fp64_values(form):
    hh = hierarchy(form, 32, 0, True)
    o = oracle_hierarchy(form, 32, 0, True)
    r = rhs_vector(19, hh.A[0].shape[0])
    ref = o.apply(r)
    err32 = energy_error(o.A[0], EmulatedVcycle(hh, policy_fp32).apply(r), ref)
    errw = energy_error(o.A[0], EmulatedVcycle(hh, policy_wide).apply(r), ref)
    errdf = energy_error(o.A[0], EmulatedVcycle(hh, policy_df).apply(r), ref)
    assert err32 >= 1e-2, err32      # measured 3.1e-2 (H(curl)), 3.6e-2 (H(div))
    assert errw <= 1e-3, errw        # measured 4.9e-5, 4.4e-5
    assert errdf <= 1e-3, errdf      # double-float residuals: measured 4.9e-5, 4.4e-5


def _df_case(form):
    """A near-gradient (curl) field on a contrast operator: most of A x cancels."""
    hh = hierarchy(form, 8, 2, True)
    A = hh.A[0].to_scipy().tocsr()
    G = hh.G[0].to_scipy().tocsr()
    rng = np.random.default_rng(23)
    x = (G @ rng.uniform(-1, 1, G.shape[1]) + 1e-3 * rng.uniform(-1, 1, A.shape[1])).astype(np.float32)
    b = rng.uniform(-1e-3, 1e-3, A.shape[0]).astype(np.float32)
    # reference in extended precision, row by row
    Al = A.astype(np.longdouble)
    exact = b.astype(np.longdouble) - Al @ x.astype(np.longdouble)
    w = np.diff(A.indptr)
    scale = np.abs(b).astype(np.float64) + abs(A) @ np.abs(x).astype(np.float64)
    bound = 0.5 * np.finfo(np.float32).eps * np.abs(exact.astype(np.float64)) + (w * w + 4 * w + 8) * 2.0 ** -48 * scale
    return A, x, b, exact, bound, scale


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_double_float_residual_within_its_bound(form):
    """The double-float residual (values as float pairs, exact product remainders,
    pair sums; rounded once to float32) stays within (w^2 + 4 w + 8) 2^-48 (|b| + |A||x|)
    of b - A x in extended precision on a cancelling field -- far below FP32's
    eps_32 (|b| + |A||x|), which a plain float32 product exceeds."""
    A, x, b, exact, bound, scale = _df_case(form)
    err = np.abs(resid_df(A, x, b).astype(np.longdouble) - exact).astype(np.float64)
    assert np.all(err <= bound), float((err / bound).max())
    err32 = np.abs((b - A.astype(np.float32) @ x).astype(np.longdouble) - exact).astype(np.float64)
    assert np.any(err32 > 100 * bound)       # FP32 values and sums miss it by far


@pytest.mark.parametrize("plant", ["no_low_sum", "no_low_value"])
def test_double_float_residual_planted_mistakes(plant):
    """Dropping the pair sum's low part, or the values' low halves, breaks the bound."""
    A, x, b, exact, bound, scale = _df_case("hcurl")
    if plant == "no_low_value":
        orig = fp32_emulation.split_df
        fp32_emulation.split_df = lambda v: (orig(v)[0], np.zeros(len(v), dtype=np.float32))
        try:
            y = resid_df(A, x, b)
        finally:
            fp32_emulation.split_df = orig
    else:
        sh = b.astype(np.float32).copy()      # the high parts' two-sum chain alone
        hi_all, _ = fp32_emulation.split_df(A.data)
        lens = np.diff(A.indptr)
        for k in range(int(lens.max())):
            rows = np.nonzero(lens > k)[0]
            pos = A.indptr[rows] + k
            sh[rows] = sh[rows] + (-hi_all[pos]) * x[A.indices[pos]]
        y = sh
    err = np.abs(y.astype(np.longdouble) - exact).astype(np.float64)
    assert np.any(err > 10 * bound)
