"""GPU re-setup for new coefficients (amge_update_coefficients), against the oracle
built from the generator's hierarchy for those coefficients.

A hierarchy set up by amge_setup_upload for one coefficient field is given another;
the re-assembled A_0, the Galerkin chain A_{l+1} = P_l^T A_l P_l (Section 3.2.1) and the
derived smoother data on the GPU must give the V-cycle and PCG solve of a fresh setup
with the new field: one V-cycle within the single-vector bound, PCG within one
iteration and 1e-9 of the oracle's solution; the FP32 V-cycle reaches 1e-8.  Updating
back to the first field restores its solution to that tolerance (the first operators
came from the host's Galerkin products, the restored ones from the GPU's).  Hierarchies uploaded as CSR levels have
no assembly data and are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


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


def _check_solves(amge, h, hh, b, label):
    from oracle import OracleHierarchy, pcg

    o = OracleHierarchy.from_hierarchy(hh)
    z = torch.empty_like(dev(b))
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP64)
    ref = o.apply(b)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref), label
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, _, ok = pcg(o, b, rtol=1e-8)
    assert st == amge.AMGE_OK and ok, label
    assert abs(info[0]["iters"] - it_o) <= 1, (label, info[0]["iters"], it_o)
    xg = host(x)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), label
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE)
    assert st == amge.AMGE_OK and info[0]["iters"] <= it_o + 3, label
    assert np.linalg.norm(b - o.A[0] @ host(x)) <= 1e-8 * np.linalg.norm(b), label
    return xg


@pytest.mark.parametrize("form,n", [("hcurl", 16), ("hdiv", 16), ("hcurl", 24)])
def test_update_coefficients_matches_fresh_setup(amge, form, n):
    from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector
    from paper_2107_05613_gb300.inputs.rng import block_coefficients, workload_coefficients

    b1, a1 = workload_coefficients(n, True, 2107056139)
    b2 = block_coefficients(n, 4, -2.0, 2.0, 2107056140)
    a2 = block_coefficients(n, 8, -1.0, 1.0, 2107056141)
    h = amge.amge_setup_upload(form, n, 0, b1, a1)
    rhs = rhs_vector(2107056142, h.n)
    x1 = _check_solves(amge, h, build_hierarchy(form, n, 0, b1, a1), rhs, "first field")
    amge.amge_update_coefficients(h, b2, a2)
    _check_solves(amge, h, build_hierarchy(form, n, 0, b2, a2), rhs, "updated field")
    amge.amge_update_coefficients(h, b1, a1)
    x1b = _check_solves(amge, h, build_hierarchy(form, n, 0, b1, a1), rhs, "first field again")
    # the first operators came from the host's Galerkin products, these from the GPU's
    # (another summation order): the solutions agree to the parity tolerance
    assert np.linalg.norm(x1b - x1) <= 1e-9 * np.linalg.norm(x1)
    h.free()


def test_update_refusals(amge):
    from paper_2107_05613_gb300.inputs import build_hierarchy

    hh = build_hierarchy("hcurl", 8, 2)
    h = amge.amge_upload_levels(hh)
    with pytest.raises(amge.AmgeError):                # CSR-level upload: no assembly data
        amge.amge_update_coefficients(h, None, None)
    h.free()
    h = amge.amge_setup_upload("hcurl", 8, 2)
    bad = np.ones(6 * 8 ** 3)
    bad[3] = -1.0
    with pytest.raises(amge.AmgeError):
        amge.amge_update_coefficients(h, bad, None)
    amge.amge_update_coefficients(h, None, None)       # all ones: the problem it was made for
    h.free()
