"""The coarsest-level solve that allocates no device memory, through the C ABI.

Callers that may not have the library allocate device memory while they solve
(a latency-critical loop that cannot afford cudaMalloc's device-wide
synchronisation, or a framework that owns every device byte through its own pool)
call amge_coarse_solve_noalloc with their own vectors only; its intermediate
vector lives in a fixed 4096-double device array.  It must give what the regular
coarsest solve (amge_apply with AMGE_OP_COARSE) gives, call after call.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test.
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


def _hier(form, n, levels):
    from paper_2107_05613_gb300.inputs import build_hierarchy
    from paper_2107_05613_gb300.inputs.rng import workload_coefficients

    beta, alpha = workload_coefficients(n, True, 2107056130)
    return build_hierarchy(form, n, num_levels=levels, beta=beta, alpha=alpha)


def test_noalloc_matches_regular_coarse_solve_on_consecutive_calls(amge):
    hh = _hier("hcurl", 16, 2)                      # coarsest level: 1,944 edge dofs
    h = amge.amge_upload_levels(hh)
    Ac = hh.A[-1].to_scipy().toarray()
    nc = Ac.shape[0]
    # same tolerance as the coarsest-solve parity tests: the solve's forward error scale
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(Ac))
    rng = np.random.default_rng(11)
    bs = [torch.from_numpy(rng.uniform(-1, 1, nc)).cuda() for _ in range(2)]
    z_ref = [torch.empty_like(b) for b in bs]
    z_new = [torch.full_like(b, float("nan")) for b in bs]
    for b, z in zip(bs, z_ref):
        amge.amge_apply(h, amge.AMGE_OP_COARSE, 0, b, z, amge.AMGE_FP64)
    torch.cuda.synchronize()
    # two calls in a row on one stream with no synchronisation between them: the
    # second call's first product overwrites the shared array only after the first
    # call's second product has read it (stream order)
    for b, z in zip(bs, z_new):
        amge.amge_coarse_solve_noalloc(h, b, z)
    torch.cuda.synchronize()
    for call in range(2):
        zr, zn = z_ref[call].cpu().numpy(), z_new[call].cpu().numpy()
        assert np.all(np.isfinite(zn)), call
        assert np.linalg.norm(zn - zr) <= tol * np.linalg.norm(zr), call
    h.free()


def test_noalloc_rejects_coarse_levels_beyond_its_array(amge):
    hh = _hier("hcurl", 8, 1)                       # one level: 4,184 dofs > 4,096
    h = amge.amge_upload_levels(hh)
    b = torch.zeros(hh.A[0].shape[0], dtype=torch.float64, device="cuda")
    z = torch.empty_like(b)
    with pytest.raises(amge.AmgeError) as e:
        amge.amge_coarse_solve_noalloc(h, b, z)
    assert e.value.status == amge.AMGE_EINVAL
    assert "at most 4096" in amge.amge_last_error()
    h.free()
