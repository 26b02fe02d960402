"""The CUDA path on hierarchies enriched by approximation targets (Sections 3.3.1,
3.3.3): the enlarged last prolongator and its Galerkin coarsest matrix go through the
same upload, V-cycle and PCG as any hierarchy, and match the FP64 oracle on them --
the V-cycle within the coarse-solve bound, the FP64 PCG within one iteration and 1e-9
(relative L2) in the solution, the FP32 V-cycle's PCG to a true FP64 residual of 1e-8.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
CASES = [("hcurl", 8, 2, 1), ("hdiv", 8, 2, 1), ("hcurl", 16, 3, 1), ("hdiv", 16, 3, 1), ("hcurl", 8, 2, 2),
         ("hdiv", 8, 2, 2)]


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


@functools.lru_cache(maxsize=None)
def _hier(form, n, L, deg=1):
    from paper_2107_05613_gb300.inputs import build_hierarchy, workload_coefficients

    beta, alpha = workload_coefficients(n, True, 13)
    return build_hierarchy(form, n, L, beta, alpha, targets=deg)


@functools.lru_cache(maxsize=None)
def _oracle(form, n, L, deg=1):
    from oracle import OracleHierarchy

    return OracleHierarchy.from_hierarchy(_hier(form, n, L, deg))


_up = {}


def _upload(amge, form, n, L, deg=1):
    if (form, n, L, deg) not in _up:
        _up[(form, n, L, deg)] = amge.amge_upload_levels(_hier(form, n, L, deg))
    return _up[(form, n, L, deg)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("form,n,L,deg", CASES)
def test_vcycle_on_enriched_hierarchy_matches_oracle(amge, form, n, L, deg):
    from paper_2107_05613_gb300.inputs import rhs_vector

    assert _hier(form, n, L, deg).diagnostics["target_functions"] > 0
    h, o = _upload(amge, form, n, L, deg), _oracle(form, n, L, deg)
    r = rhs_vector(41, o.A[0].shape[0])
    z = torch.empty_like(dev(r))
    amge.amge_vcycle(h, dev(r), z, 1, amge.AMGE_FP64)
    ref = o.apply(r)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("form,n,L,deg", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_on_enriched_hierarchy(amge, form, n, L, deg, prec):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h, o = _upload(amge, form, n, L, deg), _oracle(form, n, L, deg)
    b = rhs_vector(43, o.A[0].shape[0])
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8,
                                   precision=amge.AMGE_FP64 if prec == 0 else amge.AMGE_FP32_VCYCLE)
    assert st == amge.AMGE_OK
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    xo, it_o, _, ok = pcg(o, b, rtol=1e-8)
    assert ok
    if prec == 0:
        assert abs(info[0]["iters"] - it_o) <= 1
        assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    else:
        assert info[0]["iters"] <= it_o + 3, (info[0]["iters"], it_o)


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_problem_setup_with_targets_matches_oracle(amge, form):
    """The C-ABI problem-level setup with AMGE_SETUP_TARGETS builds the same enriched
    hierarchy: its V-cycle matches the oracle of the Python-built one."""
    from paper_2107_05613_gb300.inputs import rhs_vector, workload_coefficients

    n, L = 8, 2
    beta, alpha = workload_coefficients(n, True, 13)
    h = amge.amge_setup_upload(form, n, L, beta, alpha, targets=True)
    o = _oracle(form, n, L)
    assert h.n == o.A[0].shape[0]
    r = rhs_vector(47, h.n)
    z = torch.empty_like(dev(r))
    amge.amge_vcycle(h, dev(r), z, 1, amge.AMGE_FP64)
    ref = o.apply(r)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    assert np.linalg.norm(host(z) - ref) <= tol * np.linalg.norm(ref)
