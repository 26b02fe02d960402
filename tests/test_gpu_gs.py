"""GPU parity of the Gauss-Seidel hybrid smoother (the smoother of the paper's runs,
Section 5.1: two symmetric Gauss-Seidel steps for the primary and for the auxiliary
smoothing of eq. 4.1, here in a multicolour order) against the oracle's, through the
C ABI.

Both sides colour the same patterns with the same greedy rule, so the row orders and
the operations agree; the sums within a row differ in order, so results agree to
rounding: one V-cycle within the single-vector bound max(1e-11, 10 eps kappa(A_L)),
PCG within one iteration and 1e-9 of the oracle's solution.  Gauss-Seidel on the
finest level only (l1-Jacobi below) is checked the same way; the graph-driven loop
equals the host-launched one; FP32 V-cycles and blocks are refused.
"""
import numpy as np
import pytest

from conftest import hierarchy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
GS_CASES = [("hcurl", 8, 2, None), ("hdiv", 8, 2, None), ("hcurl", 16, 2, None), ("hdiv", 24, 3, None),
            ("hcurl", 8, 4, None), ("hcurl", 24, 3, 1)]


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


def _setup(amge, form, n, L, gs_levels):
    from oracle import OracleHierarchy

    hh = hierarchy(form, n, L, True)
    h = amge.amge_upload_levels(hh)
    amge.amge_set_smoother(h, amge.AMGE_SMOOTHER_SYM_GS, 2, 64 if gs_levels is None else gs_levels)
    o = OracleHierarchy.from_hierarchy(hh, smoother="gs", sweeps=2, gs_levels=gs_levels)
    return h, o


@pytest.mark.parametrize("form,n,L,gs_levels", GS_CASES)
def test_gs_vcycle_and_pcg_match_oracle(amge, form, n, L, gs_levels):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h, o = _setup(amge, form, n, L, gs_levels)
    r = rhs_vector(97, o.A[0].shape[0])
    z = torch.empty_like(dev(r))
    amge.amge_vcycle(h, dev(r), z, 1, amge.AMGE_FP64)
    ref = o.apply(r)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref)
    b = rhs_vector(101, o.A[0].shape[0])
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, _, ok = pcg(o, b, rtol=1e-8)
    assert st == amge.AMGE_OK and ok
    assert abs(info[0]["iters"] - it_o) <= 1, (info[0]["iters"], it_o)
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    h.free()


def test_gs_graph_equals_host_loop_and_refusals(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h, _ = _setup(amge, "hcurl", 16, 2, None)
    b = dev(rhs_vector(103, h.n))
    xg, xh = torch.empty_like(b), torch.empty_like(b)
    amge.amge_set_graphs(h, True)
    st_g, ig = amge.amge_pcg_solve(h, b, xg)
    amge.amge_set_graphs(h, False)
    st_h, ih = amge.amge_pcg_solve(h, b, xh)
    amge.amge_set_graphs(h, True)
    assert st_g == st_h == amge.AMGE_OK and ig[0]["iters"] == ih[0]["iters"]
    assert torch.equal(xg, xh)
    with pytest.raises(amge.AmgeError):
        amge.amge_pcg_solve(h, b, xg, precision=amge.AMGE_FP32_VCYCLE)
    B = dev(rhs_vector(107, h.n, 4))
    with pytest.raises(amge.AmgeError):
        amge.amge_pcg_solve(h, B, torch.empty_like(B), nrhs=4)
    # back to l1-Jacobi: FP32 and blocks run again, with the earlier results
    amge.amge_set_smoother(h, amge.AMGE_SMOOTHER_L1_JACOBI, 1, 0)
    st, info = amge.amge_pcg_solve(h, b, xg, precision=amge.AMGE_FP32_VCYCLE)
    assert st == amge.AMGE_OK and info[0]["true_relres"] <= 1e-8
    with pytest.raises(amge.AmgeError):
        amge.amge_set_smoother(h, 7, 2, 1)
    h.free()
