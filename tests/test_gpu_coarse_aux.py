"""GPU parity of the auxiliary-space coarsest solver (amge_set_coarse_solver with
AMGE_COARSE_AUX; Sections 4.2 and 5.1, eq. 4.2) against the oracle's
AuxSpaceCoarseSolver on the same generated hierarchies (built with all spaces).

The GPU's generalized inverses of the auxiliary matrices come from pivoted Cholesky,
the oracle's from eigendecompositions (pseudo-inverses); on the range the
preconditioner uses they agree to rounding (CPU check: V-cycles 1e-12 apart).  So
the V-cycle matches the oracle's to 1e-9 relative, PCG within one iteration and its
solution to 1e-9; the FP32 V-cycle with the same coarsest solver reaches the FP64
tolerance within the oracle's iterations + 3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _setup(amge, form, n, L):
    from oracle import OracleHierarchy
    from paper_2107_05613_gb300.inputs import build_hierarchy
    from paper_2107_05613_gb300.inputs.rng import workload_coefficients

    b, a = workload_coefficients(n, True, 11)
    hh = build_hierarchy(form, n, L, b, a, all_spaces=True)
    h = amge.amge_upload_levels(hh)
    amge.amge_set_coarse_solver(h, amge.AMGE_COARSE_AUX, 5, *amge.amge_coarse_aux_inputs(hh))
    return hh, h, OracleHierarchy.from_hierarchy(hh, coarse="aux")


@pytest.mark.parametrize("form,n,L", [("hcurl", 8, 2), ("hdiv", 8, 2), ("hcurl", 16, 2), ("hdiv", 16, 3),
                                       ("hcurl", 8, 1)])
def test_aux_coarse_vcycle_and_pcg_match_oracle(amge, form, n, L):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    hh, h, o = _setup(amge, form, n, L)
    b = rhs_vector(31, h.n)
    z = torch.empty(h.n, dtype=torch.float64, device="cuda")
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP64)
    ref = o.apply(b)
    assert np.linalg.norm(host(z) - ref) <= 1e-9 * np.linalg.norm(ref)
    x = torch.empty_like(z)
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, _, ok = pcg(o, b, rtol=1e-8)
    assert st == amge.AMGE_OK and ok and abs(info[0]["iters"] - it_o) <= 1, (info[0]["iters"], it_o)
    assert np.linalg.norm(host(x) - xo) <= 1e-9 * np.linalg.norm(xo)
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE)
    assert st == amge.AMGE_OK and info[0]["iters"] <= it_o + 3
    assert np.linalg.norm(b - o.A[0] @ host(x)) <= 1e-8 * np.linalg.norm(b)
    # back to the dense solve: the default solver's results again
    amge.amge_set_coarse_solver(h, amge.AMGE_COARSE_DENSE)
    from oracle import OracleHierarchy
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP64)
    ref_d = OracleHierarchy.from_hierarchy(hh).apply(b)
    assert np.linalg.norm(host(z) - ref_d) <= 1e-9 * np.linalg.norm(ref_d)
    h.free()


def test_aux_coarse_refusals(amge):
    from paper_2107_05613_gb300.inputs import build_hierarchy

    hh = build_hierarchy("hdiv", 8, 2, all_spaces=True)
    h = amge.amge_upload_levels(hh)
    pihat, D, inner = amge.amge_coarse_aux_inputs(hh)
    for bad in [dict(solver=2), dict(solver=1, iters=0), dict(solver=1, pihat_inner=None)]:
        kw = dict(solver=1, iters=5, pihat=pihat, D=D, pihat_inner=inner)
        kw.update(bad)
        with pytest.raises(amge.AmgeError):
            amge.amge_set_coarse_solver(h, kw["solver"], kw["iters"], kw["pihat"], kw["D"], kw["pihat_inner"])
    with pytest.raises(amge.AmgeError):                 # wrong row count
        amge.amge_set_coarse_solver(h, 1, 5, hh.pihat[0][2], D, inner)
    h.free()


def test_aux_coarse_after_coefficient_update(amge):
    """A hierarchy made by the problem-level setup takes the auxiliary-space solver (the
    interpolations do not depend on the coefficients); a coefficient update drops it for
    the dense solve, and setting it again forms its matrices from the new A_L."""
    from oracle import OracleHierarchy
    from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector
    from paper_2107_05613_gb300.inputs.rng import block_coefficients, workload_coefficients

    n = 8
    b1, a1 = workload_coefficients(n, True, 11)
    b2 = block_coefficients(n, 4, -2.0, 2.0, 12)
    h = amge.amge_setup_upload("hcurl", n, 2, b1, a1)
    hh1 = build_hierarchy("hcurl", n, 2, b1, a1, all_spaces=True)
    hh2 = build_hierarchy("hcurl", n, 2, b2, a1, all_spaces=True)
    rhs = rhs_vector(41, h.n)
    z = torch.empty(h.n, dtype=torch.float64, device="cuda")

    def check(o):
        amge.amge_vcycle(h, dev(rhs), z, 1, amge.AMGE_FP64)
        ref = o.apply(rhs)
        assert np.linalg.norm(host(z) - ref) <= 1e-9 * np.linalg.norm(ref)

    amge.amge_set_coarse_solver(h, amge.AMGE_COARSE_AUX, 5, *amge.amge_coarse_aux_inputs(hh1))
    check(OracleHierarchy.from_hierarchy(hh1, coarse="aux"))
    amge.amge_update_coefficients(h, b2, a1)
    check(OracleHierarchy.from_hierarchy(hh2))                 # dense again
    amge.amge_set_coarse_solver(h, amge.AMGE_COARSE_AUX, 5, *amge.amge_coarse_aux_inputs(hh2))
    check(OracleHierarchy.from_hierarchy(hh2, coarse="aux"))
    h.free()
