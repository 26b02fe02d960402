"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py
times: H(curl) and H(div) on 64^3 Kuhn-split cubes with beta contrast 1e6, 4 levels,
the same seeded coefficients and right-hand side as the benchmark, autotuned kernels,
streamed level-0 operators, the captured PCG loop.

* every level-0 product, sampled: 4,096 random rows plus the last 64 rows (the ragged
  last slice) of y = M x against the oracle's rows, within the bound of one CSR
  product, 2 (nnz_i + 1) eps (|M||x|)_i; for A G the stored product's entry rounding
  and its dropped cancellation residue (64 eps (|A||G||x|)_i) come on top;
* the same samples for the FP32 copies (streamed FP32 kernels), with the FP32 bound of
  the small cases, and for the FP32 V-cycle's FP64-operator product (AMGE_OP_A_WIDE)
  on gradient (curl) fields, with its bound (eps32/2 |y|_i + 2 (nnz_i + 1) eps64
  (|A||x|)_i against the exact product of the FP32-rounded input);
* one FP64 V-cycle, whole vector, against the oracle's: relative L2 within the bound
  of the small cases, max(1e-11, 10 eps kappa(A_L)); one FP32 V-cycle within 1e-3 in
  the energy norm;
* the FP64 PCG solve of the benchmark: iterations within +-1 of the oracle's, the
  true relative residual of the GPU solution, recomputed on the host, <= 1e-8, and the
  solution within 1e-9 (relative L2) of the oracle's;
* the FP32-V-cycle PCG solve of the benchmark: true relative residual <= 1e-8,
  iterations within 3 of the FP64 oracle's, solution within 1e-7 of the oracle's
  (the distance is printed).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


_cache = {}
_oracle_solutions = {}


def workload(amge, name):
    """(uploaded hierarchy, oracle hierarchy, right-hand side) of a benchmark workload."""
    if name not in _cache:
        import bench
        from oracle import OracleHierarchy

        for k in list(_cache):  # one full-size hierarchy on the device at a time
            del _cache[k]
        torch.cuda.synchronize()
        hh, b = bench.make_workload(bench.WORKLOADS[name])
        _cache[name] = (amge.amge_upload_levels(hh), OracleHierarchy.from_hierarchy(hh), np.asarray(b).ravel())
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def sample_rows(n, rng):
    return np.unique(np.concatenate([rng.choice(n, size=min(n, 4096), replace=False), np.arange(max(n - 64, 0), n)]))


class pinned_level0:
    """Pin every sliced-ELL level-0 operator of h (both precisions) to one kernel code
    for the block, restoring the autotuned choices afterwards."""

    def __init__(self, amge, h, code):
        self.amge, self.h, self.code = amge, h, code

    def __enter__(self):
        self.saved = self.amge.amge_autotune_report(self.h)
        if self.code != "tuned":
            for (l, p, o), v in self.saved.items():
                if l == 0 and (v == 0 or v >= 100):
                    self.amge.amge_set_kernel(self.h, l, p, o, self.code)

    def __exit__(self, *exc):
        for (l, p, o), v in self.saved.items():
            if v >= 0:
                self.amge.amge_set_kernel(self.h, l, p, o, v)


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernels", ["tuned", 1000, 1200, 3000, 1600, 1700, 1900, 2000])
def test_level0_products_sampled(amge, name, prec, kernels):
    """The level-0 products on the autotuned kernels, on the sliced-ELL kernels that
    prefetch each slice into L2 with one and two warps per slice, and on the one that
    stages each warp's slices into shared memory by bulk copies."""
    h, o, _ = workload(amge, name)
    with pinned_level0(amge, h, kernels):
        _level0_products(amge, h, o, name, prec)


def _level0_products(amge, h, o, name, prec):
    rep = amge.amge_autotune_report(h)
    rng = np.random.default_rng(7 + prec)
    eps = EPS64 if prec == 0 else EPS32
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
        amge.amge_apply(h, op, 0, dev(x), y, prec)
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
        # FP32: the rounding of operator entries and input on top of the product's own
        slack = 2 * k * eps * bound + (0 if prec == 0 else 2 * eps * bound)
        err = np.abs(host(y)[rows] - ref)
        assert np.all(err <= slack + 1e-300), (name, prec, op, float((err / (bound + 1e-300)).max()))


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
@pytest.mark.parametrize("kernels", ["tuned", 1000, 1200])
@pytest.mark.parametrize("arith", [1, 0])
def test_level0_wide_product_sampled(amge, name, kernels, arith):
    """The level-0 product of the FP32 V-cycle's corrected residuals, in double-float
    (1) and FP64 (0) arithmetic, on a near-gradient field (most of A x cancels)."""
    h, o, _ = workload(amge, name)
    try:
        amge.amge_set_wide_arith(h, arith)
        with pinned_level0(amge, h, kernels):
            _level0_wide(amge, h, o, name, arith)
    finally:
        amge.amge_set_wide_arith(h, amge.AMGE_WIDE_DF)


def _level0_wide(amge, h, o, name, arith):
    rng = np.random.default_rng(9)
    A, G = o.A[0], o.G[0]
    x = G @ rng.uniform(-1, 1, G.shape[1]) + 1e-3 * rng.uniform(-1, 1, A.shape[1])
    x32 = x.astype(np.float32).astype(np.float64)
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    amge.amge_apply(h, amge.AMGE_OP_A_WIDE, 0, dev(x), y, amge.AMGE_FP32_VCYCLE)
    rows = sample_rows(A.shape[0], rng)
    Ar = A[rows]
    ref = Ar @ x32
    w = np.diff(Ar.indptr)
    if arith == amge.AMGE_WIDE_FP64:
        bound = 0.5 * EPS32 * np.abs(ref) + 2 * (w + 1) * EPS64 * (abs(Ar) @ abs(x32))
    else:  # double-float: 48-bit values, pair sums (see the parity test's wide_bound)
        bound = 0.5 * EPS32 * np.abs(ref) + (w * w + 4 * w + 8) * 2.0 ** -48 * (abs(Ar) @ abs(x32))
    err = np.abs(host(y)[rows] - ref)
    assert np.all(err <= bound + 1e-300), (name, float((err / (bound + 1e-300)).max()))


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("base,code", [(0, 3000), (0, 1600), (200, 1800), (0, 2000)])
def test_level0_bulk_staged_equals_one_warp(amge, name, prec, base, code):
    """At full size, in the launch configuration of the timed solves: the level-0
    operators on the bulk-staged kernel (code 3000) or with 16-bit column offsets
    (1600, where built: H(curl)) give the V-cycle and the PCG solve of the one-warp
    sliced-ELL kernel (code 0) bit for bit, and those with 16-bit offsets on two warps
    per slice (1800) those of the two-warp kernel (200)."""
    h, o, b = workload(amge, name)
    bd = dev(b)
    res = []
    for c in (base, code):
        with pinned_level0(amge, h, c):
            z, x = torch.empty_like(bd), torch.empty_like(bd)
            amge.amge_vcycle(h, bd, z, 1, prec)
            st, info = amge.amge_pcg_solve(h, bd, x, rtol=1e-8, precision=prec)
            assert st == amge.AMGE_OK and not amge.amge_wait_status(h)
            res.append((z, x, info[0]["iters"]))
    (z0, x0, i0), (z1, x1, i1) = res
    assert torch.equal(z0, z1) and torch.equal(x0, x1) and i0 == i1


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_vcycle_full_size(amge, name):
    h, o, b = workload(amge, name)
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP64)
    ref = o.apply(b)
    tol = max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))
    rel = np.linalg.norm(host(z) - ref) / np.linalg.norm(ref)
    assert rel <= tol, (name, rel, tol)
    amge.amge_vcycle(h, dev(b), z, 1, amge.AMGE_FP32_VCYCLE)
    d = host(z) - ref
    A = o.A[0]
    err = np.sqrt((d @ (A @ d)) / (ref @ (A @ ref)))
    print(f"{name}: FP32 V-cycle energy-norm distance to the FP64 oracle cycle {err:.2e}")
    assert err <= 1e-3, (name, err)


def oracle_solution(name, o, b):
    from oracle import pcg

    if name not in _oracle_solutions:
        _oracle_solutions[name] = pcg(o, b, rtol=1e-8)
    return _oracle_solutions[name]


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_pcg_full_size(amge, name):
    h, o, b = workload(amge, name)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, rr_o, ok_o = oracle_solution(name, o, b)
    assert st == amge.AMGE_OK and ok_o
    assert abs(info[0]["iters"] - it_o) <= 1, (info[0]["iters"], it_o)
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"{name}: FP64 solution vs oracle, relative L2 {rel:.2e}")
    assert rel <= 1e-9, (name, rel)


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_pcg_full_size_fp32_vcycle(amge, name):
    h, o, b = workload(amge, name)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE)
    xo, it_o, _, ok_o = oracle_solution(name, o, b)
    assert st == amge.AMGE_OK and ok_o, (st, info)
    assert info[0]["iters"] <= it_o + 3, (info[0]["iters"], it_o)
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"{name}: FP32-V-cycle solution vs FP64 oracle, relative L2 {rel:.2e}, "
          f"{info[0]['iters']} iterations (oracle {it_o})")
    assert rel <= 1e-7, (name, rel)


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_pcg_full_size_fp32_vcycle_block(amge, name):
    """Blocks of right-hand sides under the 1e6 contrast with the FP32 V-cycle: its
    corrected residuals in double-float arithmetic (an all-FP32 block cycle stagnates
    here, as the single-vector one did).  Four columns: the workload's right-hand side
    (checked against the oracle's solution) and three more; every column reaches the
    FP64 tolerance within the oracle's iteration count + 3."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h, o, b = workload(amge, name)
    nrhs = 4
    B = np.stack([b] + [rhs_vector(900 + k, b.size) for k in range(1, nrhs)], axis=1)
    X = torch.empty((b.size, nrhs), dtype=torch.float64, device="cuda")
    st, info = amge.amge_pcg_solve(h, dev(B), X, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE, nrhs=nrhs)
    xo, it_o, _, ok_o = oracle_solution(name, o, b)
    assert st == amge.AMGE_OK and ok_o, (st, info)
    Xg = host(X)
    for k in range(nrhs):
        assert info[k]["status"] == amge.AMGE_OK and info[k]["iters"] <= it_o + 3, (k, info[k], it_o)
        assert np.linalg.norm(B[:, k] - o.A[0] @ Xg[:, k]) <= 1e-8 * np.linalg.norm(B[:, k]), k
    rel = np.linalg.norm(Xg[:, 0] - xo) / np.linalg.norm(xo)
    print(f"{name}: FP32-V-cycle block solve, column 0 vs FP64 oracle, relative L2 {rel:.2e}, "
          f"iterations {[i['iters'] for i in info]} (oracle {it_o})")
    assert rel <= 1e-7, (name, rel)


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_pcg_product_forms_equal(amge, name):
    """The PCG product q = A_0 p with 32-bit columns, with 16-bit column offsets and
    per-slice L2 prefetch (where A_0 has them) and with 32-bit columns and the prefetch
    form the same sums: identical solves."""
    h, o, b = workload(amge, name)
    bd = dev(b)
    saved, us = amge.amge_pcg_kernel(h)
    res = []
    try:
        for code in (0, 1700, 1000):
            amge.amge_pcg_kernel(h, code)
            x = torch.empty_like(bd)
            st, info = amge.amge_pcg_solve(h, bd, x, rtol=1e-8, precision=amge.AMGE_FP64)
            assert st == amge.AMGE_OK
            res.append((x, info[0]["iters"]))
    finally:
        amge.amge_pcg_kernel(h, saved)
    print(f"{name}: PCG product {us} us (32-bit / 16-bit + prefetch / 32-bit + prefetch), kept {saved}")
    for x, it in res[1:]:
        assert torch.equal(res[0][0], x) and res[0][1] == it


@pytest.mark.parametrize("name", ["hcurl64", "hdiv64"])
def test_double_float_forms_equal(amge, name):
    """The FP32 V-cycle's double-float product with 32-bit columns (one warp per slice)
    and with 16-bit column offsets, without and with the L2 prefetch, form the same
    sums: identical V-cycles and FP32-V-cycle solves."""
    h, o, b = workload(amge, name)
    bd = dev(b)
    saved, us = amge.amge_df_form(h, 0)
    rep = amge.amge_autotune_report(h)
    res = []
    try:
        amge.amge_set_kernel(h, 0, "fp64", "A", 0)     # the 32-bit form's warps per slice: one
        for form in (0, 1, 2):
            got, _ = amge.amge_df_form(h, 0, form)
            z, x = torch.empty_like(bd), torch.empty_like(bd)
            amge.amge_vcycle(h, bd, z, 1, amge.AMGE_FP32_VCYCLE)
            st, info = amge.amge_pcg_solve(h, bd, x, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE)
            assert st == amge.AMGE_OK
            res.append((got, z, x, info[0]["iters"]))
    finally:
        amge.amge_df_form(h, 0, saved)
        amge.amge_set_kernel(h, 0, "fp64", "A", rep[(0, "fp64", "A")])
    print(f"{name}: double-float level-0 product {us} us (32-bit / 16-bit / 16-bit + prefetch), kept {saved}")
    for got, z, x, it in res[1:]:
        assert torch.equal(z, res[0][1]) and torch.equal(x, res[0][2]) and it == res[0][3], got
