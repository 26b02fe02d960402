"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py
times: H(curl) and H(div) on 64^3 Kuhn-split cubes with beta contrast 1e6, 4 levels,
the same seeded coefficients and right-hand side as the benchmark, autotuned kernels,
streamed level-0 operators, the captured PCG loop.

* every level-0 product, sampled: 4,096 random rows plus the last 64 rows (the ragged
  last slice) of y = M x against the oracle's rows, within the bound of one CSR
  product, 2 (nnz_i + 1) eps (|M||x|)_i; for A G the stored product's entry rounding
  and its dropped cancellation residue (64 eps (|A||G||x|)_i) come on top;
* one FP64 V-cycle, whole vector, against the oracle's: relative L2 within the bound
  of the small cases, max(1e-11, 10 eps kappa(A_L));
* the FP64 PCG solve of the benchmark: iterations within +-1 of the oracle's and the
  true relative residual of the GPU solution, recomputed on the host, <= 1e-8.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


_cache = {}


def workload(amge, name):
    """(uploaded hierarchy, oracle hierarchy, right-hand side) of a benchmark workload."""
    if name not in _cache:
        import bench
        from oracle import OracleHierarchy

        for k in list(_cache):  # one full-size hierarchy on the device at a time
            del _cache[k]
        torch.cuda.synchronize()
        hh, b = bench.make_workload(bench.WORKLOADS[name])
        _cache[name] = (amge.amge_setup_upload(hh), OracleHierarchy.from_hierarchy(hh), np.asarray(b).ravel())
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def sample_rows(n, rng):
    return np.unique(np.concatenate([rng.choice(n, size=min(n, 4096), replace=False), np.arange(max(n - 64, 0), n)]))


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_level0_products_sampled(amge, name):
    h, o, _ = workload(amge, name)
    rep = amge.amge_autotune_report(h)
    rng = np.random.default_rng(7)
    A, P, G = o.A[0], o.P[0], o.G[0]
    ops = {amge.AMGE_OP_A: A, amge.AMGE_OP_P: P, amge.AMGE_OP_PT: P.T.tocsr(), amge.AMGE_OP_G: G,
           amge.AMGE_OP_GT: G.T.tocsr()}
    if rep[(0, "fp64", "AG")] >= 0:
        ops[amge.AMGE_OP_AG] = None
    for op, M in ops.items():
        ncols = G.shape[1] if op == amge.AMGE_OP_AG else M.shape[1]
        nrows = A.shape[0] if op == amge.AMGE_OP_AG else M.shape[0]
        x = rng.uniform(-1, 1, ncols)
        y = torch.empty(nrows, dtype=torch.float64, device="cuda")
        amge.amge_apply(h, op, 0, dev(x), y, amge.AMGE_FP64)
        rows = sample_rows(nrows, rng)
        if op == amge.AMGE_OP_AG:
            Ar = A[rows]
            ref = Ar @ (G @ x)
            bound = abs(Ar) @ (abs(G) @ abs(x))
            k = np.diff(Ar.indptr) * np.diff(G.indptr).max() + 1 + 64
        else:
            Mr = M[rows]
            ref = Mr @ x
            bound = abs(Mr) @ abs(x)
            k = np.diff(Mr.indptr) + 1
        err = np.abs(host(y)[rows] - ref)
        assert np.all(err <= 2 * k * EPS64 * bound + 1e-300), (name, op, float((err / (bound + 1e-300)).max()))


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_vcycle_full_size(amge, name):
    h, o, b = workload(amge, name)
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP64)
    ref = o.apply(b)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    rel = np.linalg.norm(host(z) - ref) / np.linalg.norm(ref)
    assert rel <= tol, (name, rel, tol)


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_pcg_full_size(amge, name):
    from oracle import pcg

    h, o, b = workload(amge, name)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, rr_o, ok_o = pcg(o, b, rtol=1e-8)
    assert st == amge.AMGE_OK and ok_o
    assert abs(info[0]["iters"] - it_o) <= 1, (info[0]["iters"], it_o)
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
