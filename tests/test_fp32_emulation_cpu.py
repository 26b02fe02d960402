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
from fp32_emulation import EmulatedVcycle, energy_error, policy_fp32, policy_fp64, policy_wide
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
    assert err32 >= 1e-2, err32      # measured 3.1e-2 (H(curl)), 3.6e-2 (H(div))
    assert errw <= 1e-3, errw        # measured 4.9e-5, 3.3e-5
