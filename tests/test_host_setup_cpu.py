"""CPU tests of the library's host preparation (csrc/amge_host_setup.cpp), compiled
with a test-only C shim (tests/host_setup_shim.cpp); no GPU.  Each step is checked
against an independent computation (scipy / numpy) on small matrices:

* CSR validation rejects every malformed input it documents;
* the stored zeros of an input operator are dropped, nothing else;
* transpose, l1 row sums and the aux l1 row sums of G^T A G;
* the A G product: equal to scipy's, with the cancellation residue
  |c_ij| <= 64 eps (|A||G|)_ij dropped and everything above it kept;
* the coarsest Cholesky factor, its inverse and A^{-1};
* the sliced-ELL layout (slices of 32 rows sorted by length inside windows, pairs,
  padding, sign-coded columns): every row reconstructs exactly.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS = np.finfo(np.float64).eps
PAD = -(2 ** 31)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA runtime header is not available")
    out = str(tmp_path_factory.mktemp("shim") / "libhostshim.so")
    subprocess.run([cxx, "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2107_05613_gb300", "csrc"),
                    "-I", cuda_inc, os.path.join(ROOT, "tests", "host_setup_shim.cpp"),
                    os.path.join(ROOT, "paper_2107_05613_gb300", "csrc", "amge_host_setup.cpp"), "-o", out],
                   check=True, capture_output=True)
    L = ctypes.CDLL(out)
    vp, i32, i64, dp, ip = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    for name, args, res in [
        ("shim_check_csr", [i32, i32, i64, ip, ip, dp], i32),
        ("shim_to_host", [i32, i32, i64, ip, ip, dp], vp),
        ("shim_csr", [i32, i32, ip, ip, dp], vp),
        ("shim_csr_free", [vp], None),
        ("shim_csr_shape", [vp, ip], None),
        ("shim_csr_copy", [vp, ip, ip, dp], None),
        ("shim_transpose", [vp], vp),
        ("shim_product", [vp, vp], vp),
        ("shim_l1", [vp, dp], None),
        ("shim_aux_l1", [vp, vp, vp, dp], None),
        ("shim_coarse", [vp, dp, dp, dp], i32),
        ("shim_sell", [vp, i32, i32], vp),
        ("shim_sell_free", [vp], None),
        ("shim_sell_info", [vp, ip], None),
        ("shim_sell_copy", [vp, ip, ip, ip, dp], None),
        ("shim_sell16", [vp, ip, ip, ip], i32),
        ("shim_ginv", [i32, dp, dp, ctypes.c_double], i32),
        ("shim_error", [], ctypes.c_char_p),
    ]:
        f = getattr(L, name)
        f.argtypes, f.restype = args, res
    return L


def _ptr(a):
    return a.ctypes.data


def to_shim(lib, M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    rp, ci, v = (np.ascontiguousarray(M.indptr, np.int32), np.ascontiguousarray(M.indices, np.int32),
                 np.ascontiguousarray(M.data, np.float64))
    return lib.shim_csr(M.shape[0], M.shape[1], _ptr(rp), _ptr(ci), _ptr(v))


def from_shim(lib, h):
    info = np.zeros(3, np.int64)
    lib.shim_csr_shape(h, _ptr(info))
    nr, nc, nnz = (int(x) for x in info)
    rp, ci, v = np.zeros(nr + 1, np.int32), np.zeros(max(nnz, 1), np.int32), np.zeros(max(nnz, 1))
    lib.shim_csr_copy(h, _ptr(rp), _ptr(ci), _ptr(v))
    lib.shim_csr_free(h)
    return sp.csr_matrix((v[:nnz], ci[:nnz], rp), shape=(nr, nc))


def random_csr(rng, nr, nc, density, integer=False):
    M = sp.random(nr, nc, density=density, random_state=rng, format="csr")
    if integer:
        M.data = rng.integers(-3, 4, M.nnz).astype(np.float64)
        M.eliminate_zeros()
    else:
        M.data = rng.uniform(-1, 1, M.nnz)
    M.sort_indices()
    return M


def test_check_csr_rejects_malformed(lib):
    rp = np.array([0, 2, 3], np.int32)
    ci = np.array([0, 2, 1], np.int32)
    v = np.array([1.0, 2.0, 3.0])
    assert lib.shim_check_csr(2, 3, 3, _ptr(rp), _ptr(ci), _ptr(v)) == 1
    bad = [
        (np.array([0, 2, 3], np.int32), np.array([2, 0, 1], np.int32), v, "not strictly increasing"),
        (rp, np.array([0, 3, 1], np.int32), v, "out of range"),
        (rp, np.array([0, -1, 1], np.int32), v, "out of range"),
        (np.array([0, 3, 2], np.int32), ci, v, "span"),
        (np.array([1, 2, 3], np.int32), ci, v, "span"),
        (rp, ci, np.array([1.0, np.nan, 3.0]), "non-finite"),
        (rp, ci, np.array([1.0, np.inf, 3.0]), "non-finite"),
    ]
    for r, c, x, msg in bad:
        assert lib.shim_check_csr(2, 3, 3, _ptr(r), _ptr(c), _ptr(x)) == 0
        assert msg in lib.shim_error().decode(), lib.shim_error()


def test_to_host_drops_stored_zeros_only(lib):
    rp = np.array([0, 3, 3, 6], np.int32)
    ci = np.array([0, 1, 4, 0, 2, 3], np.int32)
    v = np.array([0.0, -2.5, -0.0, 1e-300, 0.0, 7.0])
    M = from_shim(lib, lib.shim_to_host(3, 5, 6, _ptr(rp), _ptr(ci), _ptr(v)))
    assert M.nnz == 3
    assert list(M.indptr) == [0, 1, 1, 3]
    assert list(M.indices) == [1, 0, 3]
    assert list(M.data) == [-2.5, 1e-300, 7.0]


def test_transpose_and_l1_sums(lib):
    rng = np.random.default_rng(1)
    M = random_csr(rng, 57, 41, 0.15)
    T = from_shim(lib, lib.shim_transpose(to_shim(lib, M)))
    R = M.T.tocsr()
    R.sort_indices()
    assert (T.indptr == R.indptr).all() and (T.indices == R.indices).all() and (T.data == R.data).all()
    h = to_shim(lib, M)
    out = np.zeros(M.shape[0])
    lib.shim_l1(h, _ptr(out))
    lib.shim_csr_free(h)
    assert np.allclose(out, abs(M).sum(axis=1).A1, rtol=1e-15, atol=0)


def test_aux_l1_sums_equal_those_of_gtag(lib):
    rng = np.random.default_rng(2)
    A = random_csr(rng, 40, 40, 0.2, integer=True)
    A = (A + A.T).tocsr()
    G = random_csr(rng, 40, 17, 0.1, integer=True)
    ha, hg, hgt = to_shim(lib, A), to_shim(lib, G), to_shim(lib, G.T.tocsr())
    out = np.zeros(G.shape[1])
    lib.shim_aux_l1(ha, hg, hgt, _ptr(out))
    for h in (ha, hg, hgt):
        lib.shim_csr_free(h)
    ref = abs((G.T @ A @ G).tocsr()).sum(axis=1).A1   # integer data: every sum exact
    assert (out == ref).all()


def test_product_matches_scipy_without_cancellation(lib):
    rng = np.random.default_rng(3)
    A = random_csr(rng, 60, 50, 0.1)
    A.data = np.abs(A.data) + 0.5                  # positive terms: no cancellation
    B = random_csr(rng, 50, 30, 0.1)
    B.data = np.abs(B.data) + 0.5
    C = from_shim(lib, lib.shim_product(to_shim(lib, A), to_shim(lib, B)))
    R = (A @ B).tocsr()
    R.sort_indices()
    assert (C.indptr == R.indptr).all() and (C.indices == R.indices).all()
    assert np.allclose(C.data, R.data, rtol=8 * EPS, atol=0)


def test_product_drops_cancellation_residue_only(lib):
    # row 0: 1 - (1 - 2^-52) = 2^-52, i.e. 1.1e-16 of the terms' magnitude: residue;
    # row 1: 1 - (1 - 2^-40) = 2^-40, 4.5e-13 of it: genuine, kept;
    # row 2: an exact zero; row 3: a plain entry.
    A = sp.csr_matrix(np.array([[1.0, -(1.0 - 2.0 ** -52), 0.0],
                                [1.0, -(1.0 - 2.0 ** -40), 0.0],
                                [2.0, -2.0, 0.0],
                                [0.0, 0.0, 3.0]]))
    G = sp.csr_matrix(np.array([[1.0], [1.0], [1.0]]))
    C = from_shim(lib, lib.shim_product(to_shim(lib, A), to_shim(lib, G)))
    assert list(np.diff(C.indptr)) == [0, 1, 0, 1]
    assert C.data[0] == 2.0 ** -40 and C.data[1] == 3.0
    # the rule on a larger operator: kept entries above 64 eps of their magnitudes,
    # dropped ones at or below it, and the kept ones equal to scipy's
    rng = np.random.default_rng(4)
    A = random_csr(rng, 80, 80, 0.1)
    G = random_csr(rng, 80, 30, 0.05, integer=True)
    G.data = np.sign(G.data)
    C = from_shim(lib, lib.shim_product(to_shim(lib, A), to_shim(lib, G)))
    R = (A @ G).tocsr()
    M = (abs(A) @ abs(G)).tocsr()
    Rd, Md, Cd = R.toarray(), M.toarray(), C.toarray()
    kept = Cd != 0
    assert np.all(np.abs(Rd[kept] - Cd[kept]) <= 8 * EPS * Md[kept])
    assert np.all(np.abs(Rd[~kept]) <= 64 * EPS * Md[~kept] + 8 * EPS * Md[~kept])
    assert np.all(np.abs(Cd[kept]) > 64 * EPS * Md[kept])


def test_coarse_factor_and_inverse(lib):
    rng = np.random.default_rng(5)
    n = 37
    X = rng.standard_normal((n, n))
    A = X @ X.T + n * np.eye(n)
    h = to_shim(lib, sp.csr_matrix(A))
    L, LT, I = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    assert lib.shim_coarse(h, _ptr(L), _ptr(LT), _ptr(I)) == 1
    lib.shim_csr_free(h)
    assert np.allclose(np.triu(L, 1), 0) and (LT == L.T).all()
    assert np.allclose(L @ A @ L.T, np.eye(n), atol=1e-12)
    assert (I == I.T).all()
    assert np.allclose(I, np.linalg.inv(A), rtol=1e-10, atol=1e-14)
    h = to_shim(lib, sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]])))   # indefinite
    assert lib.shim_coarse(h, _ptr(L), _ptr(LT), _ptr(I)) == 0
    lib.shim_csr_free(h)


def sell_rows(lib, M, sigma, allow_unit):
    h = to_shim(lib, M)
    s = lib.shim_sell(h, sigma, int(allow_unit))
    lib.shim_csr_free(h)
    info = np.zeros(3, np.int64)
    lib.shim_sell_info(s, _ptr(info))
    ns, stored, unit = (int(x) for x in info)
    sptr, srow = np.zeros(ns + 1, np.int64), np.zeros(ns * 32, np.int32)
    ci, v = np.zeros(max(stored, 1), np.int32), np.zeros(max(stored, 1))
    lib.shim_sell_copy(s, _ptr(sptr), _ptr(srow), _ptr(ci), _ptr(v))
    lib.shim_sell_free(s)
    return ns, sptr, srow, ci, v, bool(unit)


@pytest.mark.parametrize("sigma", [32, 1024])
def test_sliced_ell_reconstructs_every_row(lib, sigma):
    rng = np.random.default_rng(6)
    nr = 1100                                   # a ragged last slice, more than one window
    lens = rng.integers(0, 12, nr)
    lens[5] = 0
    rows, cols, vals = [], [], []
    for i, l in enumerate(lens):
        c = np.sort(rng.choice(300, size=l, replace=False))
        rows += [i] * l
        cols += list(c)
        vals += list(rng.uniform(0.5, 1.5, l) * rng.choice([-1, 1], l))
    M = sp.csr_matrix((vals, (rows, cols)), shape=(nr, 300))
    M.sort_indices()
    ns, sptr, srow, ci, v, unit = sell_rows(lib, M, sigma, False)
    assert not unit and ns == (nr + 31) // 32
    assert (sptr % 64 == 0).all()
    assert sorted(srow[srow >= 0]) == list(range(nr)) and (srow[nr:] == -1).all()
    for w0 in range(0, nr, sigma):                 # rows sorted by length inside windows
        L = [lens[r] for r in srow[w0:min(nr, w0 + sigma)]]
        assert all(a >= b for a, b in zip(L, L[1:]))
    for s in range(ns):
        w = (sptr[s + 1] - sptr[s]) // 32
        for j in range(32):
            r = srow[s * 32 + j]
            if r < 0:
                continue
            at = [sptr[s] + (k // 2) * 64 + 2 * j + (k & 1) for k in range(w)]
            lo, hi = M.indptr[r], M.indptr[r + 1]
            l = hi - lo
            assert list(ci[at[:l]]) == list(M.indices[lo:hi]) and list(v[at[:l]]) == list(M.data[lo:hi])
            assert (v[at[l:]] == 0).all()          # padding: value 0 at a valid column
            assert ((ci[at[l:]] >= 0) & (ci[at[l:]] < 300)).all()


def test_sliced_ell_sign_coded(lib):
    rng = np.random.default_rng(7)
    G = random_csr(rng, 200, 90, 0.04, integer=True)
    G.data = np.sign(G.data)
    G.eliminate_zeros()
    ns, sptr, srow, ci, v, unit = sell_rows(lib, G, 1024, True)
    assert unit
    for s in range(ns):
        w = (sptr[s + 1] - sptr[s]) // 32
        for j in range(32):
            r = srow[s * 32 + j]
            if r < 0:
                continue
            lo, hi = G.indptr[r], G.indptr[r + 1]
            got = [ci[sptr[s] + (k // 2) * 64 + 2 * j + (k & 1)] for k in range(w)]
            dec = [(c, 1.0) if c >= 0 else (~c, -1.0) for c in got[:hi - lo]]
            assert dec == list(zip(G.indices[lo:hi], G.data[lo:hi]))
            assert all(c == PAD for c in got[hi - lo:])
    # a matrix with another value is not sign-coded
    G2 = G.copy()
    G2.data[0] = 2.0
    assert not sell_rows(lib, G2, 1024, True)[5]


def _sell16(lib, M, sigma=1024):
    h = to_shim(lib, M)
    s = lib.shim_sell(h, sigma, 0)
    lib.shim_csr_free(h)
    info = np.zeros(3, np.int64)
    lib.shim_sell_info(s, _ptr(info))
    ns, stored = int(info[0]), int(info[1])
    sptr, srow = np.zeros(ns + 1, np.int64), np.zeros(ns * 32, np.int32)
    ci, v = np.zeros(max(stored, 1), np.int32), np.zeros(max(stored, 1))
    lib.shim_sell_copy(s, _ptr(sptr), _ptr(srow), _ptr(ci), _ptr(v))
    bases = np.zeros(ns * 32, np.int32)
    c16 = np.zeros(max(stored // 2, 1), np.uint32)
    nb = np.zeros(1, np.int64)
    mode = lib.shim_sell16(s, _ptr(bases), _ptr(c16), _ptr(nb))
    lib.shim_sell_free(s)
    return mode, ns, sptr, srow, ci, bases[:nb[0]], c16


def _check16(mode, ns, sptr, srow, ci, bases, c16):
    """Every live lane's decoded columns equal the 32-bit ones."""
    for s in range(ns):
        w = (sptr[s + 1] - sptr[s]) // 64
        for j in range(32):
            if srow[s * 32 + j] < 0:
                continue
            base = bases[s] if mode == 1 else bases[s * 32 + j]
            for k in range(w):
                p = sptr[s] + k * 64 + 2 * j
                u = int(c16[p // 2])
                assert (base + (u & 0xFFFF), base + (u >> 16)) == (ci[p], ci[p + 1])


def test_sliced_ell_16bit_columns(lib):
    """16-bit column offsets: one base per slice where every slice spans fewer than
    65,536 columns; one per row where only the rows do (a slice gathering rows far
    apart); none where a row spans more."""
    rng = np.random.default_rng(8)
    n = 200_000
    # banded rows: every slice narrow
    rows = np.repeat(np.arange(3000), 5)
    cols = np.minimum(rows * 10 + rng.integers(0, 5000, rows.size), n - 1)
    M = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(3000, n))
    M.sum_duplicates()
    mode, *rest = _sell16(lib, M)
    assert mode == 1
    _check16(mode, *rest)
    # rows narrow, but row i starts at column 6,000 (i mod 32): every 32-row slice spans
    # about 246,000 columns
    rows = np.repeat(np.arange(3000), 4)
    cols = (rows % 32) * 6000 + rng.integers(0, 60000, rows.size)
    M = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(3000, 260_000))
    M.sum_duplicates()
    mode, *rest = _sell16(lib, M)
    assert mode == 2
    _check16(mode, *rest)
    # a row spanning more than 65,535 columns: not built
    M = sp.csr_matrix((np.ones(2), ([0, 0], [0, 70000])), shape=(40, n))
    assert _sell16(lib, M)[0] == 0


@pytest.mark.parametrize("rank", [40, 33, 1])
def test_generalized_inverse(lib, rank):
    """Pivoted-Cholesky generalized inverse of a positive semi-definite matrix:
    symmetric, S G S = S, the rank found; the inverse itself for a nonsingular S."""
    rng = np.random.default_rng(rank)
    n = 40
    B = rng.standard_normal((n, rank)) * np.exp(rng.uniform(-3, 3, rank))
    S = B @ B.T
    G = np.zeros((n, n))
    r = lib.shim_ginv(n, _ptr(np.ascontiguousarray(S)), _ptr(G), 1e-12)
    assert r == rank
    assert np.abs(G - G.T).max() == 0
    assert np.abs(S @ G @ S - S).max() <= 1e-8 * np.abs(S).max()
    if rank == n:
        assert np.abs(G @ S - np.eye(n)).max() <= 1e-6
