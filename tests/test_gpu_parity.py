"""GPU parity of the CUDA solve path against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic):
  * single operators (one CSR product, FP64): |y - y_ref|_i <= 2 (nnz_i + 1) eps64 (|M||x|)_i,
    twice the bound of a sum of nnz_i products (both sides round, in different orders);
    FP32 copies: the same with eps32 plus the rounding of operator and input to FP32.
  * one V-cycle (FP64): relative L2 <= max(1e-11, 10 eps64 kappa(A_L)); the coarsest
    solve is backward stable on both sides, so its forward difference is of order
    kappa(A_L) eps64 (the GPU multiplies by the inverse Cholesky factor, the oracle
    substitutes); the other steps add O(nnz eps64).
  * PCG (FP64): iterations within +-1 of the oracle, solution relative L2 <= 1e-9,
    true relative residual <= 1e-8.
  * the FP32 V-cycle's FP64-operator product (AMGE_OP_A_WIDE): against the exact
    product of the FP32-rounded input, eps32/2 |y_ref|_i (the final rounding) plus
    2 (nnz_i + 1) eps64 (|M||x|)_i -- tight enough to catch a product that sums in
    FP32 on inputs whose product cancels (gradient fields).
  * one FP32 V-cycle: energy-norm distance to the FP64 oracle cycle <= 1e-3 (a fixed
    bound; the CPU emulation of the same steps measures 5e-5 at 32^3 and 9e-5 at 64^3
    under the 1e6 coefficient contrast).
  * PCG with the FP32 V-cycle: true FP64 relative residual <= 1e-8, iterations within
    3 of the FP64 oracle's, and the solution within 1e-7 (relative L2) of the FP64
    oracle's.
"""
import numpy as np
import pytest

from conftest import hierarchy, oracle_hierarchy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def amge():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import amge as mod

    return mod


_uploaded = {}


def upload(amge, form, n, L, contrast=True):
    key = (form, n, L, contrast)
    if key not in _uploaded:
        _uploaded[key] = amge.amge_upload_levels(hierarchy(form, n, L, contrast))
    return _uploaded[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [("hcurl", 8, 2), ("hdiv", 8, 2), ("hcurl", 16, 2), ("hcurl", 24, 3), ("hdiv", 24, 3), ("hcurl", 8, 4)]


def _coarse_tol(o):
    return max(1e-11, 10 * EPS64 * np.linalg.cond(o.A[-1].toarray()))


class pinned_kernels:
    """Run a block with every operator of h on one kernel (0 = sliced ELL, k = vector
    CSR with k lanes per row); the autotuned choices are restored afterwards."""

    def __init__(self, amge, h, lanes):
        self.amge, self.h, self.lanes = amge, h, lanes

    def __enter__(self):
        self.saved = self.amge.amge_autotune_report(self.h)
        if self.lanes != "tuned":
            for (l, p, o), v in self.saved.items():
                if v >= 0:
                    self.amge.amge_set_kernel(self.h, l, p, o, self.lanes)
        return self

    def __exit__(self, *exc):
        for (l, p, o), v in self.saved.items():
            if v >= 0:
                self.amge.amge_set_kernel(self.h, l, p, o, v)


@pytest.mark.parametrize("form,n,L", CASES)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("lanes", ["tuned", 0, 200, 800, 4, 32, 3000, 1600, 1700, 1800, 1900, 2000])
def test_single_operators(amge, form, n, L, prec, lanes):
    """Every stored product on every smoothing level, on each kernel: sliced ELL with
    one, two and eight warps per slice (sign-coded for the +-1 incidences G), with the
    slices staged into shared memory by bulk copies (3000), with 16-bit column offsets
    (1600), vector CSR with 4 and 32 lanes per row, and the autotuned choice."""
    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    rng = np.random.default_rng(n * 7 + L)
    eps = EPS64 if prec == 0 else EPS32
    rep = amge.amge_autotune_report(h)
    with pinned_kernels(amge, h, lanes):
        for l in range(L - 1):
            ops = {amge.AMGE_OP_A: o.A[l], amge.AMGE_OP_P: o.P[l], amge.AMGE_OP_PT: o.P[l].T.tocsr(),
                   amge.AMGE_OP_G: o.G[l], amge.AMGE_OP_GT: o.G[l].T.tocsr()}
            if rep[(l, "fp64", "AG")] >= 0:
                ops[amge.AMGE_OP_AG] = (o.A[l] @ o.G[l]).tocsr()
            for op, M in ops.items():
                x = rng.uniform(-1, 1, M.shape[1])
                y = torch.empty(M.shape[0], dtype=torch.float64, device="cuda")
                amge.amge_apply(h, op, l, dev(x), y, prec)
                ref = M @ x
                nnz = np.diff(M.indptr)
                if op == amge.AMGE_OP_AG:
                    # the stored A G carries the rounding of its entries (sums of
                    # products of A and G) on top of the product's own
                    bound = abs(o.A[l]) @ (abs(o.G[l]) @ abs(x))
                    nnz = nnz + np.diff(o.A[l].indptr).max() * np.diff(o.G[l].indptr).max()
                else:
                    bound = abs(M) @ abs(x)
                slack = 2 * (nnz + 1) * eps * bound + (0 if prec == 0 else 2 * eps * bound)
                err = np.abs(host(y) - ref)
                assert np.all(err <= slack + 1e-300), (l, op, float((err / (bound + 1e-300)).max()))


@pytest.mark.parametrize("form,prec,gsep", [("hcurl", 0, 200), ("hcurl", 1, 200), ("hdiv", 1, 2000)])
@pytest.mark.parametrize("ag", [0, 200, 400, 800, 1600])
def test_fused_aux_correction_equals_separate_products(amge, form, prec, gsep, ag):
    """With G on the one-warp and A G on a sliced-ELL kernel (1, 2, 4 or 8 warps per
    slice, or 16-bit columns) the V-cycle forms x += G y and r -= (A G) y (and the final
    z = x + G y + m^-1 (r - (A G) y)) in one pass with that many warps per slice: H(curl)
    with the gradient's two entries per row, H(div)'s FP32 V-cycle with the curl's three
    (finest level) or four (coarse levels).  Forcing G onto another kernel runs the
    separate products -- for H(curl) the two-warp kernel (its rows are one entry pair),
    for H(div) the grid-stride one-warp kernel (code 2000) -- whose sums are formed in
    the same order: the V-cycles must agree exactly."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, 24, 3)
    rep = amge.amge_autotune_report(h)
    pname = "fp64" if prec == 0 else "fp32"
    b = dev(rhs_vector(73, h.n))
    zf, zs = torch.empty_like(b), torch.empty_like(b)
    levels = [l for l in range(2) if rep[(l, pname, "AG")] >= 0]
    assert 0 in levels
    saved = {l: (rep[(l, pname, "G")], rep[(l, pname, "AG")]) for l in levels}
    try:
        for l in levels:
            amge.amge_set_kernel(h, l, pname, "G", 0)
            amge.amge_set_kernel(h, l, pname, "AG", ag)
        amge.amge_vcycle(h, b, zf, precision=prec)
        for l in levels:
            amge.amge_set_kernel(h, l, pname, "G", gsep)
        amge.amge_vcycle(h, b, zs, precision=prec)
    finally:
        for l, (g, ag) in saved.items():
            amge.amge_set_kernel(h, l, pname, "G", g)
            amge.amge_set_kernel(h, l, pname, "AG", ag)
    torch.cuda.synchronize()
    assert torch.isfinite(zf).all() and torch.equal(zf, zs)


@pytest.mark.parametrize("form,n,L", [("hcurl", 8, 2), ("hdiv", 24, 3), ("hcurl", 24, 3)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("base,code", [(0, 3000), (0, 1600), (200, 1800), (0, 2000)])
def test_bulk_staged_equals_one_warp_kernel(amge, form, n, L, prec, base, code):
    """The bulk-staged product (code 3000: each warp's slices copied into shared memory
    two ahead), the 16-bit-column product (1600) and the grid-stride product (2000:
    each warp walks many slices, loading the next one's entries ahead) form every row's
    sum in the order of the one-warp sliced-ELL kernel (code 0), the two-warp
    16-bit-column product (1800) in that of the two-warp kernel (200): products,
    V-cycles and graph-driven PCG solves are identical, and no staged copy's wait runs
    out."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    b = dev(rhs_vector(83, h.n))
    res = {}
    for c in (base, code):
        with pinned_kernels(amge, h, c):
            out = []
            for l in range(L - 1):
                shapes = {amge.AMGE_OP_A: o.A[l].shape, amge.AMGE_OP_P: o.P[l].shape,
                          amge.AMGE_OP_PT: o.P[l].T.shape, amge.AMGE_OP_G: o.G[l].shape,
                          amge.AMGE_OP_GT: o.G[l].T.shape}
                for op, (nr, nc) in shapes.items():
                    x = dev(np.random.default_rng(l * 10 + op).uniform(-1, 1, nc))
                    y = torch.empty(nr, dtype=torch.float64, device="cuda")
                    amge.amge_apply(h, op, l, x, y, prec)
                    out.append(y)
            z, x = torch.empty_like(b), torch.empty_like(b)
            amge.amge_vcycle(h, b, z, precision=prec)
            st, info = amge.amge_pcg_solve(h, b, x, precision=prec)
            assert st == amge.AMGE_OK
            res[c] = (out, z, x, info[0]["iters"])
            assert not amge.amge_wait_status(h)
    (o0, z0, x0, i0), (o1, z1, x1, i1) = res[base], res[code]
    assert all(torch.equal(a, c) for a, c in zip(o0, o1))
    assert torch.equal(z0, z1) and torch.equal(x0, x1) and i0 == i1


@pytest.mark.parametrize("prec", [0, 1])
def test_dependent_launch_does_not_change_results(amge, prec):
    """Programmatic dependent launch only changes when blocks are scheduled: the
    V-cycle and the graph-driven PCG give identical results with it on and off."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    b = dev(rhs_vector(79, hierarchy("hcurl", 24, 3, True).A[0].shape[0]))
    out = []
    try:
        for on in (True, False):
            amge.amge_set_dependent_launch(on)
            h = amge.amge_upload_levels(hierarchy("hcurl", 24, 3, True))
            rep = amge.amge_autotune_report(h)
            out.append((h, rep))
    finally:
        amge.amge_set_dependent_launch(True)
    (h1, rep1), (h0, rep0) = out
    for (l, p, o), v in rep1.items():      # same kernels on both
        if v >= 0:
            amge.amge_set_kernel(h0, l, p, o, v)
    for l in range(2):                     # and the same double-float forms and PCG product
        amge.amge_df_form(h0, l, amge.amge_df_form(h1, l)[0])
    amge.amge_pcg_kernel(h0, amge.amge_pcg_kernel(h1)[0])
    amge.amge_set_dependent_launch(False)
    try:
        z0, x0 = torch.empty_like(b), torch.empty_like(b)
        amge.amge_vcycle(h0, b, z0, precision=prec)
        st0, i0 = amge.amge_pcg_solve(h0, b, x0, precision=prec)
    finally:
        amge.amge_set_dependent_launch(True)
    z1, x1 = torch.empty_like(b), torch.empty_like(b)
    amge.amge_vcycle(h1, b, z1, precision=prec)
    st1, i1 = amge.amge_pcg_solve(h1, b, x1, precision=prec)
    torch.cuda.synchronize()
    assert st0 == st1 == amge.AMGE_OK and i0[0]["iters"] == i1[0]["iters"]
    assert torch.equal(z0, z1) and torch.equal(x0, x1)


def test_set_kernel_rebuilds_graph_and_rejects_bad_input(amge):
    """A pinned kernel choice takes effect in the captured PCG graph (rebuilt on the
    next solve): results move by rounding only and the solve still matches the oracle."""
    from oracle.amge_oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 24, 3)
    o = oracle_hierarchy("hcurl", 24, 3, True)
    b_np = rhs_vector(71, h.n)
    x_ref, it_ref, _, _ = pcg(o, b_np, rtol=1e-8, maxit=500)
    b = dev(b_np)
    for lanes in ("tuned", 0, 400, 4):
        with pinned_kernels(amge, h, lanes):
            x = torch.empty_like(b)
            st, info = amge.amge_pcg_solve(h, b, x)
            assert st == amge.AMGE_OK and abs(info[0]["iters"] - it_ref) <= 1
            xs = host(x)
            assert np.linalg.norm(xs - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    for bad in [(5, 0, 0, 0), (0, 2, 0, 0), (0, 0, 6, 0), (0, 0, 0, 3), (0, 0, 0, 64)]:
        with pytest.raises(amge.AmgeError):
            amge.amge_set_kernel(h, *bad)
    # A G is stored only for one pre- and one post-smoothing step (the updates
    # r -= (A G) y replace those steps' residuals)
    hd = amge.amge_upload_levels(hierarchy("hdiv", 24, 3, True), nu_pre=2, nu_post=2)
    assert all(v < 0 for (l, p, o), v in amge.amge_autotune_report(hd).items() if o == "AG")
    with pytest.raises(amge.AmgeError):
        amge.amge_set_kernel(hd, 0, 0, "AG", 0)
    with pytest.raises(amge.AmgeError):
        amge.amge_apply(hd, amge.AMGE_OP_AG, 0, b[: 10], b[: 10], 0)
    # H(div) with one step each: A C (= alpha M C) is stored for the FP32 V-cycle
    rep = amge.amge_autotune_report(upload(amge, "hdiv", 24, 3))
    assert rep[(0, "fp32", "AG")] >= 0


def _hybrid_step_bound(o, b):
    """Elementwise bound on |computed - exact| of one hybrid step from x0 = 0 in FP64,
    propagated through x = b/m, r = b - A x, y = (G^T r)/m_aux, x += G y.  Both sides
    derive m and m_aux themselves: m_aux sums |G^T A G| whose entries cancel the
    (Du, Dv) part, so each entry carries up to K eps (|G^T||A||G|) of rounding
    (K = terms per entry), which enters y relatively."""
    A, G = o.A[0], o.G[0]
    GT = G.T.tocsr()
    aA, aG, aGT = abs(A), abs(G), abs(GT)
    nA, nG, nGT = np.diff(A.indptr), np.diff(G.indptr), np.diff(GT.indptr)
    K = nGT.max() * nA.max() * nG.max()
    x = b / o.m[0]
    r = b - A @ x
    y = (G.T @ r) / o.m_aux[0]
    dmaux = K * EPS64 * (aGT @ (aA @ (aG @ np.ones(G.shape[1])))) / o.m_aux[0]
    ex = (nA + 2) * EPS64 * abs(x)
    er = aA @ ex + (nA + 1) * EPS64 * (abs(b) + aA @ abs(x))
    ey = (aGT @ er + (nGT + 1) * EPS64 * (aGT @ abs(r))) / o.m_aux[0] + (dmaux + 2 * EPS64) * abs(y)
    return ex + aG @ ey + (nG + 1) * EPS64 * (abs(x) + aG @ abs(y))


@pytest.mark.parametrize("form,n,L", CASES)
def test_smoother_step_and_coarse_solve(amge, form, n, L):
    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    b = np.random.default_rng(5).uniform(-1, 1, o.A[0].shape[0])
    y = torch.empty_like(dev(b))
    amge.amge_apply(h, amge.AMGE_OP_SMOOTH_PRE, 0, dev(b), y, 0)
    ref = o.hybrid(0, np.zeros_like(b), b)
    # both sides round: twice the one-sided propagated bound
    assert np.all(np.abs(host(y) - ref) <= 2 * _hybrid_step_bound(o, b))
    bc = np.random.default_rng(6).uniform(-1, 1, o.A[-1].shape[0])
    z = torch.empty_like(dev(bc))
    amge.amge_apply(h, amge.AMGE_OP_COARSE, 0, dev(bc), z, 0)
    ref = o.coarse_solve(bc)
    assert np.linalg.norm(host(z) - ref) <= _coarse_tol(o) * np.linalg.norm(ref)


@pytest.mark.parametrize("form,n,L", CASES)
def test_vcycle_fp64_matches_oracle(amge, form, n, L):
    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    from paper_2107_05613_gb300.inputs import rhs_vector

    r = rhs_vector(17, o.A[0].shape[0])
    z = torch.empty_like(dev(r))
    amge.amge_vcycle(h, dev(r), z, 1, amge.AMGE_FP64)
    ref = o.apply(r)
    assert np.linalg.norm(host(z) - ref) <= _coarse_tol(o) * np.linalg.norm(ref)


FP32_CASES = CASES + [("hcurl", 32, 3), ("hdiv", 32, 3)]


@pytest.mark.parametrize("form,n,L", FP32_CASES)
def test_vcycle_fp32_close_to_oracle(amge, form, n, L):
    """FP32 V-cycle vs the FP64 oracle in the energy norm, under the 1e6 coefficient
    contrast: within 1e-3 (the residuals of corrected iterates run on the FP64
    operators; an all-FP32 cycle is 3e-2 off at 32^3 and 1.3e-1 at 64^3)."""
    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    from paper_2107_05613_gb300.inputs import rhs_vector

    r = rhs_vector(19, o.A[0].shape[0])
    z = torch.empty_like(dev(r))
    amge.amge_vcycle(h, dev(r), z, 1, amge.AMGE_FP32_VCYCLE)
    ref = o.apply(r)
    A = o.A[0]
    d = host(z) - ref
    err = np.sqrt((d @ (A @ d)) / (ref @ (A @ ref)))
    assert err <= 1e-3, err


def wide_bound(amge, arith, A, x32, ref):
    """Error bound of AMGE_OP_A_WIDE (y = fl32(A x) with x in FP32): the final
    rounding plus the sum's own error -- FP64 recursive summation for AMGE_WIDE_FP64;
    for AMGE_WIDE_DF the 48-bit value split, the product remainders and the
    unnormalized pair sum, at most (w^2 + 4 w + 8) 2^-48 |A| |x| for rows of w entries."""
    w = np.diff(A.indptr)
    ax = abs(A) @ abs(x32)
    if arith == amge.AMGE_WIDE_FP64:
        return 0.5 * EPS32 * np.abs(ref) + 2 * (w + 1) * EPS64 * ax
    return 0.5 * EPS32 * np.abs(ref) + (w * w + 4 * w + 8) * 2.0 ** -48 * ax


@pytest.mark.parametrize("form,n,L", FP32_CASES)
@pytest.mark.parametrize("field", ["random", "gradient"])
@pytest.mark.parametrize("arith", [1, 0])
def test_wide_product(amge, form, n, L, field, arith):
    """AMGE_OP_A_WIDE on every smoothing level: FP32 input and output, values and sums
    in double-float pairs (arith 1, the default) or FP64 (0).  On gradient (curl)
    fields, where the large-coefficient part of A x cancels, only sums carried well
    beyond FP32 meet the bound (the CPU emulation tests show FP32 failing it)."""
    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    rng = np.random.default_rng(n + 3 * L)
    try:
        amge.amge_set_wide_arith(h, arith)
        for l in range(L - 1):
            A = o.A[l]
            x = rng.uniform(-1, 1, A.shape[1])
            if field == "gradient":
                x = o.G[l] @ rng.uniform(-1, 1, o.G[l].shape[1]) + 1e-3 * x
            x32 = x.astype(np.float32).astype(np.float64)
            y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
            amge.amge_apply(h, amge.AMGE_OP_A_WIDE, l, dev(x), y, amge.AMGE_FP32_VCYCLE)
            ref = A @ x32
            bound = wide_bound(amge, arith, A, x32, ref)
            err = np.abs(host(y) - ref)
            assert np.all(err <= bound + 1e-300), (l, float((err / (bound + 1e-300)).max()))
    finally:
        amge.amge_set_wide_arith(h, amge.AMGE_WIDE_DF)
    with pytest.raises(amge.AmgeError):             # FP32 V-cycle product only
        amge.amge_apply(h, amge.AMGE_OP_A_WIDE, 0, dev(x), y, amge.AMGE_FP64)
    with pytest.raises(amge.AmgeError):
        amge.amge_set_wide_arith(h, 2)


@pytest.mark.parametrize("form,n,L", [("hcurl", 16, 2), ("hdiv", 24, 3)])
def test_wide_arith_modes_in_the_fp32_solve(amge, form, n, L):
    """Both arithmetics of the residuals of corrected iterates give FP32-V-cycle PCG
    solves that reach the FP64 tolerance in the FP64 iteration count (+3), and the
    V-cycles agree to the FP32 rounding level."""
    from oracle.amge_oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    b = rhs_vector(89, h.n)
    _, it_o, _, _ = pcg(o, b, rtol=1e-8)
    z = {}
    try:
        for arith in (amge.AMGE_WIDE_FP64, amge.AMGE_WIDE_DF):
            amge.amge_set_wide_arith(h, arith)
            x = torch.empty(h.n, dtype=torch.float64, device="cuda")
            st, info = amge.amge_pcg_solve(h, dev(b), x, precision=amge.AMGE_FP32_VCYCLE)
            assert st == amge.AMGE_OK and info[0]["iters"] <= it_o + 3, (arith, info[0]["iters"], it_o)
            assert np.linalg.norm(b - o.A[0] @ host(x)) <= 1e-8 * np.linalg.norm(b)
            z[arith] = torch.empty_like(x)
            amge.amge_vcycle(h, dev(b), z[arith], precision=amge.AMGE_FP32_VCYCLE)
    finally:
        amge.amge_set_wide_arith(h, amge.AMGE_WIDE_DF)
    d = host(z[0]) - host(z[1])
    A = o.A[0]
    ref = host(z[0])
    assert np.sqrt(d @ (A @ d)) <= 1e-4 * np.sqrt(ref @ (A @ ref))


@pytest.mark.parametrize("form,n,L", CASES)
def test_pcg_fp64_matches_oracle(amge, form, n, L):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    b = rhs_vector(23, o.A[0].shape[0])
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP64)
    xo, it_o, rr_o, ok_o = pcg(o, b, rtol=1e-8)
    assert st == amge.AMGE_OK and ok_o
    assert abs(info[0]["iters"] - it_o) <= 1
    assert info[0]["true_relres"] <= 1e-8
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)


@pytest.mark.parametrize("form,n,L", FP32_CASES)
def test_pcg_fp32_vcycle_reaches_fp64_tolerance(amge, form, n, L):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    b = rhs_vector(29, o.A[0].shape[0])
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE)
    assert st == amge.AMGE_OK
    xg = host(x)
    assert np.linalg.norm(b - o.A[0] @ xg) <= 1e-8 * np.linalg.norm(b)
    xo, it_o, _, _ = pcg(o, b, rtol=1e-8)
    assert info[0]["iters"] <= it_o + 3, (info[0]["iters"], it_o)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-7, err


def test_pcg_host_buffers(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 16, 2)
    o = oracle_hierarchy("hcurl", 16, 2, True)
    b = rhs_vector(31, o.A[0].shape[0])
    x = np.zeros_like(b)
    st, info = amge.amge_pcg_solve_host(h, b, x, rtol=1e-8)
    assert st == amge.AMGE_OK
    assert np.linalg.norm(b - o.A[0] @ x) <= 1e-8 * np.linalg.norm(b)


def test_dot_deterministic_and_exact_enough(amge):
    h = upload(amge, "hcurl", 8, 2)
    for n in (1, 1000, 1 << 20, (1 << 20) + 12345):
        rng = np.random.default_rng(n)
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        amge.amge_dot(h, dev(x), dev(y), n, out)
        a = host(out)[0]
        amge.amge_dot(h, dev(x), dev(y), n, out)
        assert host(out)[0] == a
        assert abs(a - x @ y) <= n * EPS64 * (abs(x) @ abs(y))


def test_edge_cases(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 8, 2)
    n = h.n
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    st, info = amge.amge_pcg_solve(h, torch.zeros(n, dtype=torch.float64, device="cuda"), x)
    assert st == amge.AMGE_OK and info[0]["iters"] == 0 and host(x).max() == 0
    b = dev(rhs_vector(3, n))
    st, info = amge.amge_pcg_solve(h, b, x, rtol=1e-14, maxit=2)
    assert st == amge.AMGE_ENOTCONV and info[0]["iters"] == 2 and info[0]["true_relres"] > 1e-14
    bad = b.clone()
    bad[7] = float("nan")
    st, info = amge.amge_pcg_solve(h, bad, x)
    assert st == amge.AMGE_ENONFINITE
    with pytest.raises(amge.AmgeError):
        amge.amge_vcycle(h, b, b)
    with pytest.raises(amge.AmgeError):
        amge.amge_pcg_solve(h, b, x, rtol=-1.0)


def test_one_level_hierarchy_is_direct(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    hh = hierarchy("hcurl", 4, 1, False)
    h = amge.amge_upload_levels(hh)
    A = hh.A[0].to_scipy()
    b = rhs_vector(2, A.shape[0])
    x = torch.empty_like(dev(b))
    st, info = amge.amge_pcg_solve(h, dev(b), x)
    assert st == amge.AMGE_OK and info[0]["iters"] == 1
    assert np.linalg.norm(host(x) - np.linalg.solve(A.toarray(), b)) <= 1e-10 * np.linalg.norm(host(x))


@pytest.mark.parametrize("arith", [1, 0])
def test_fp32_coarsest_solve(amge, arith):
    """The FP32 V-cycle's coarsest solve (one-level hierarchy: the V-cycle is the
    coarsest solve): FP32 input and output, the explicit inverse in double-float pairs
    with pair sums (1) or in FP64 (0), against the FP64 direct solution of the FP32
    input: within the final rounding plus the sum's error bound over n terms."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    hh = hierarchy("hcurl", 6, 1, True)
    h = amge.amge_upload_levels(hh)
    A = hh.A[0].to_scipy().toarray()
    Ainv = np.linalg.inv(A)
    b32 = rhs_vector(3, A.shape[0]).astype(np.float32).astype(np.float64)
    ref = Ainv @ b32
    n = A.shape[0]
    scale = np.abs(Ainv) @ np.abs(b32)
    # the explicit inverse itself carries the Cholesky rounding: kappa eps_64 |A^-1||b|
    kappa = np.linalg.cond(A)
    if arith == 1:
        bound = 0.5 * EPS32 * np.abs(ref) + ((n / 128 + 8) ** 2 + 300) * 2.0 ** -48 * scale + 10 * kappa * EPS64 * scale
    else:
        bound = 0.5 * EPS32 * np.abs(ref) + 2 * n * EPS64 * scale + 10 * kappa * EPS64 * scale
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    try:
        amge.amge_set_wide_arith(h, arith)
        amge.amge_vcycle(h, dev(b32), z, 1, amge.AMGE_FP32_VCYCLE)
        err = np.abs(host(z) - ref)
        assert np.all(err <= bound), float((err / bound).max())
    finally:
        h.free()


def test_solve_is_deterministic(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hdiv", 24, 3)
    b = dev(rhs_vector(37, h.n))
    x1, x2 = torch.empty_like(b), torch.empty_like(b)
    amge.amge_pcg_solve(h, b, x1)
    amge.amge_pcg_solve(h, b, x2)
    assert torch.equal(x1, x2)


# ---------------------------------------------------------------- multi-RHS blocks
@pytest.mark.parametrize("form,n,L", [("hcurl", 16, 2), ("hdiv", 24, 3)])
@pytest.mark.parametrize("nrhs", [2, 3, 8, 32])
def test_vcycle_block_matches_oracle_per_column(amge, form, n, L, nrhs):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    R = rhs_vector(41, o.A[0].shape[0], nrhs)            # [n][nrhs]
    Z = torch.empty_like(dev(R))
    amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP64)
    Zg = host(Z)
    ref = o.apply(R)
    tol = _coarse_tol(o)
    for c in range(nrhs):
        assert np.linalg.norm(Zg[:, c] - ref[:, c]) <= tol * np.linalg.norm(ref[:, c]), c


def _pin_block_forms(amge, h, nrhs, code):
    """Pin every stored block product of h to one form for nrhs columns, both
    precisions (where the sliced-ELL form applies); returns the number pinned."""
    pinned = 0
    for prec in (amge.AMGE_FP64, amge.AMGE_FP32_VCYCLE):
        codes, _ = amge.amge_autotune_report_mm(h, nrhs, prec)
        for (l, op), c in codes.items():
            if op == "coarse" or (op == "AG" and amge.amge_autotune_report(h)[(l, "fp64", "AG")] < 0):
                continue
            try:
                amge.amge_set_kernel_mm(h, l, prec, op, nrhs, code)
                pinned += 1
            except amge.AmgeError:
                assert code > 0       # only the sliced-ELL forms can be inapplicable
    return pinned


@pytest.mark.parametrize("form,n,L", [("hcurl", 16, 2), ("hdiv", 24, 3), ("hcurl", 8, 4)])
@pytest.mark.parametrize("nrhs", [4, 8, 32])
@pytest.mark.parametrize("code", [0, 1, 2])
def test_block_kernel_forms_match_oracle(amge, form, n, L, nrhs, code):
    """Every block product on one form -- CSR lane groups, sliced ELL with one or two
    16-byte vectors per lane -- through the FP64 block V-cycle, per column against the
    oracle's V-cycle (the single-vector bound); the FP32 block V-cycle on the
    constant-coefficient hierarchy within 1e-3 in the energy norm."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    for contrast in (True, False):
        hh = hierarchy(form, n, L, contrast)
        h = amge.amge_upload_levels(hh)
        o = oracle_hierarchy(form, n, L, contrast)
        R = rhs_vector(67, o.A[0].shape[0], nrhs)
        Z = torch.empty_like(dev(R))
        amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP64)      # sizes the block workspace
        assert _pin_block_forms(amge, h, nrhs, code) > 0
        ref = o.apply(R)
        if contrast:
            amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP64)
            Zg = host(Z)
            tol = _coarse_tol(o)
            for c in range(nrhs):
                assert np.linalg.norm(Zg[:, c] - ref[:, c]) <= tol * np.linalg.norm(ref[:, c]), (c, code)
        else:
            amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP32_VCYCLE)
            Zg = host(Z)
            A = o.A[0]
            for c in range(nrhs):
                d = Zg[:, c] - ref[:, c]
                err = np.sqrt((d @ (A @ d)) / (ref[:, c] @ (A @ ref[:, c])))
                assert err <= 1e-3, (c, code, err)
        h.free()


def test_block_autotune_report(amge):
    """The block tuner runs on the first block call with a column count and reports a
    choice for every stored operator, with its measured times."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = amge.amge_upload_levels(hierarchy("hcurl", 16, 3, True))
    codes, _ = amge.amge_autotune_report_mm(h, 16, amge.AMGE_FP32_VCYCLE)
    assert set(codes.values()) == {-1}
    R = dev(rhs_vector(71, h.n, 16))
    Z = torch.empty_like(R)
    amge.amge_vcycle(h, R, Z, 16, amge.AMGE_FP32_VCYCLE)
    codes, us = amge.amge_autotune_report_mm(h, 16, amge.AMGE_FP32_VCYCLE)
    for (l, op), c in codes.items():
        if op == "AG" and c == -1:
            continue
        assert c in (0, 1, 2), (l, op)
        assert us[(l, op)][c] > 0
    with pytest.raises(amge.AmgeError):             # FP32: 4 floats per vector, 12 is not a multiple of 8
        amge.amge_set_kernel_mm(h, 0, amge.AMGE_FP32_VCYCLE, "A", 12, 2)
    h.free()


@pytest.mark.parametrize("nrhs", [8, 16, 24, 32])
@pytest.mark.parametrize("code", [0, 1])
def test_block_coarse_solve_on_tensor_cores(amge, nrhs, code):
    """The coarsest product Z = A_L^{-1} B of block V-cycles on CUDA cores (code 0) and on
    the FP64 tensor cores (mma.sync m8n8k4, code 1): per column within the single-vector
    V-cycle bound of the oracle (coarsest 1,944 dofs)."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 16, 2)
    o = oracle_hierarchy("hcurl", 16, 2, True)
    R = rhs_vector(89, o.A[0].shape[0], nrhs)
    Z = torch.empty_like(dev(R))
    amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP64)
    amge.amge_set_kernel_mm(h, 0, amge.AMGE_FP64, "coarse", nrhs, code)
    amge.amge_vcycle(h, dev(R), Z, nrhs, amge.AMGE_FP64)
    codes, us = amge.amge_autotune_report_mm(h, nrhs, amge.AMGE_FP64)
    assert codes[(1, "coarse")] == code and us[(1, "coarse")][0] > 0 and us[(1, "coarse")][1] > 0
    Zg = host(Z)
    ref = o.apply(R)
    tol = _coarse_tol(o)
    for c in range(nrhs):
        assert np.linalg.norm(Zg[:, c] - ref[:, c]) <= tol * np.linalg.norm(ref[:, c]), (c, code)
    with pytest.raises(amge.AmgeError):
        amge.amge_set_kernel_mm(h, 0, amge.AMGE_FP64, "coarse", 4, 1)   # not a multiple of 8


@pytest.mark.parametrize("form,n,L,nrhs", [("hcurl", 16, 2, 4), ("hdiv", 24, 3, 5), ("hcurl", 8, 4, 32)])
def test_pcg_block_fp64_matches_oracle_per_column(amge, form, n, L, nrhs):
    from oracle import pcg
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    o = oracle_hierarchy(form, n, L, True)
    B = rhs_vector(43, o.A[0].shape[0], nrhs)
    X = torch.empty_like(dev(B))
    st, infos = amge.amge_pcg_solve(h, dev(B), X, rtol=1e-8, precision=amge.AMGE_FP64, nrhs=nrhs)
    assert st == amge.AMGE_OK
    Xg = host(X)
    for c in range(nrhs):
        xo, it_o, _, ok = pcg(o, B[:, c], rtol=1e-8)
        assert ok and abs(infos[c]["iters"] - it_o) <= 1, (c, infos[c], it_o)
        assert infos[c]["true_relres"] <= 1e-8
        assert np.linalg.norm(B[:, c] - o.A[0] @ Xg[:, c]) <= 1e-8 * np.linalg.norm(B[:, c])
        assert np.linalg.norm(Xg[:, c] - xo) <= 1e-9 * np.linalg.norm(xo)


def test_pcg_block_fp32_vcycle_and_zero_column(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 24, 3)
    o = oracle_hierarchy("hcurl", 24, 3, True)
    B = rhs_vector(47, o.A[0].shape[0], 8)
    B[:, 3] = 0.0                                        # a zero right-hand side stays zero
    X = torch.empty_like(dev(B))
    st, infos = amge.amge_pcg_solve(h, dev(B), X, rtol=1e-8, precision=amge.AMGE_FP32_VCYCLE, nrhs=8)
    assert st == amge.AMGE_OK
    Xg = host(X)
    assert infos[3]["iters"] == 0 and not Xg[:, 3].any()
    for c in (0, 1, 2, 4, 5, 6, 7):
        assert np.linalg.norm(B[:, c] - o.A[0] @ Xg[:, c]) <= 1e-8 * np.linalg.norm(B[:, c])


def test_pcg_block_host_buffers(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 16, 2)
    o = oracle_hierarchy("hcurl", 16, 2, True)
    B = rhs_vector(53, o.A[0].shape[0], 6)
    X = np.zeros_like(B)
    st, infos = amge.amge_pcg_solve_host(h, B, X, rtol=1e-8, nrhs=6)
    assert st == amge.AMGE_OK
    for c in range(6):
        assert np.linalg.norm(B[:, c] - o.A[0] @ X[:, c]) <= 1e-8 * np.linalg.norm(B[:, c])


# ---------------------------------------------------------------- graph-driven loop
@pytest.mark.parametrize("form,n,L", [("hcurl", 16, 2), ("hdiv", 24, 3), ("hcurl", 8, 4)])
@pytest.mark.parametrize("prec", [0, 1])
def test_graph_loop_equals_host_loop(amge, form, n, L, prec):
    """The WHILE-node graph and the host-launched loop run the same kernels in the
    same order: identical iterates, iteration counts and residuals."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    b = dev(rhs_vector(59, h.n))
    xg, xh = torch.empty_like(b), torch.empty_like(b)
    amge.amge_set_graphs(h, True)
    st_g, ig = amge.amge_pcg_solve(h, b, xg, precision=prec)
    amge.amge_set_graphs(h, False)
    st_h, ih = amge.amge_pcg_solve(h, b, xh, precision=prec)
    amge.amge_set_graphs(h, True)
    assert st_g == st_h == amge.AMGE_OK
    assert ig[0]["iters"] == ih[0]["iters"]
    assert ig[0]["true_relres"] == ih[0]["true_relres"]
    assert torch.equal(xg, xh)


@pytest.mark.parametrize("form,n,L,nrhs", [("hcurl", 16, 2, 8), ("hdiv", 24, 3, 5), ("hcurl", 8, 4, 32)])
@pytest.mark.parametrize("prec", [0, 1])
def test_block_graph_loop_equals_host_loop(amge, form, n, L, nrhs, prec):
    """The block PCG's WHILE-node graph runs the kernels of the host-driven block loop
    in the same order: identical iterates, per-column iteration counts and residuals
    (a zero column stays out of the iteration in both)."""
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, form, n, L)
    B = rhs_vector(83, h.n, nrhs)
    B[:, 1] = 0.0
    B = dev(B)
    Xg, Xh = torch.empty_like(B), torch.empty_like(B)
    amge.amge_set_graphs(h, True)
    st_g, ig = amge.amge_pcg_solve(h, B, Xg, precision=prec, nrhs=nrhs)
    amge.amge_set_graphs(h, False)
    st_h, ih = amge.amge_pcg_solve(h, B, Xh, precision=prec, nrhs=nrhs)
    amge.amge_set_graphs(h, True)
    assert st_g == st_h == amge.AMGE_OK
    assert [i["iters"] for i in ig] == [i["iters"] for i in ih]
    assert [i["true_relres"] for i in ig] == [i["true_relres"] for i in ih]
    assert ig[1]["iters"] == 0 and max(i["true_relres"] for i in ig) <= 1e-8
    assert torch.equal(Xg, Xh)
    for maxit in (1, 3):
        st, info = amge.amge_pcg_solve(h, B, Xg, rtol=1e-14, maxit=maxit, precision=prec, nrhs=nrhs)
        assert st == amge.AMGE_ENOTCONV
        assert all(i["iters"] == maxit for c, i in enumerate(info) if c != 1)


def test_graph_loop_maxit_and_nonfinite(amge):
    from paper_2107_05613_gb300.inputs import rhs_vector

    h = upload(amge, "hcurl", 16, 2)
    b = dev(rhs_vector(61, h.n))
    x = torch.empty_like(b)
    for maxit in (1, 2, 5):
        st, info = amge.amge_pcg_solve(h, b, x, rtol=1e-14, maxit=maxit)
        assert st == amge.AMGE_ENOTCONV and info[0]["iters"] == maxit
    bad = b.clone()
    bad[11] = float("inf")
    st, info = amge.amge_pcg_solve(h, bad, x)
    assert st == amge.AMGE_ENONFINITE
    st, info = amge.amge_pcg_solve(h, b, x)        # the hierarchy stays usable
    assert st == amge.AMGE_OK and info[0]["true_relres"] <= 1e-8


def test_autotune_report(amge):
    """Every smoothing-level operator has a kernel choice: 0 or 100 w (sliced ELL with
    w warps per slice) or a power-of-two lane count (vector CSR)."""
    h = upload(amge, "hcurl", 24, 3)
    rep = amge.amge_autotune_report(h)
    assert len(rep) == 2 * 2 * 6
    assert set(rep.values()) <= {-1, 0, 200, 400, 800, 1000, 1200, 1600, 1700, 1800, 1900, 2000, 3000, 2, 4, 8, 16,
                                 32}
    assert rep[(0, "fp64", "AG")] >= 0          # H(curl): A G is stored (much sparser than A)
    # where A G is stored the two-entry gradient G stays on code 0, so x += G y rides in
    # the fused A G pass instead of a separate product
    for (l, p, o), v in rep.items():
        if o == "AG" and v >= 0:
            assert rep[(l, p, "G")] == 0, (l, p, rep[(l, p, "G")])
