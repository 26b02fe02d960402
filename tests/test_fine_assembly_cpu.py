"""The fine assembly of A_0 written as a gather (the data of the GPU re-setup for new
coefficients), checked on the CPU against the generator's own assembly:

  * re-assembling A_0 from the gather with the generator's coefficients gives its A_0
    (the same sums in the same order; a few ulps for contraction of b K + a M);
  * with other coefficients it gives the A_0 the generator builds for them;
  * the Galerkin chain A_{l+1} = P_l^T A_l P_l of those operators gives the generator's
    coarse operators for the new coefficients, and P_l, G_l do not change (the local
    extensions of eqs. 3.6/3.8 use unweighted masses).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2107_05613_gb300.inputs import build_hierarchy
from paper_2107_05613_gb300.inputs.rng import block_coefficients, workload_coefficients

EPS = np.finfo(np.float64).eps


def _gather(asm, beta, alpha, shape, indptr, indices):
    s2 = asm["s"] ** 2
    K = asm["K"].reshape(6, s2)
    M = asm["M"].reshape(6, s2)
    c = asm["ccell"].astype(np.int64)
    terms = beta[c] * K[c % 6, asm["cidx"]] + alpha[c] * M[c % 6, asm["cidx"]]
    mags = np.abs(beta[c] * K[c % 6, asm["cidx"]]) + np.abs(alpha[c] * M[c % 6, asm["cidx"]])
    coff = asm["coff"].astype(np.int64)
    cnt = np.diff(coff)
    row = np.repeat(np.arange(cnt.size), cnt)
    val = np.bincount(row, weights=terms, minlength=cnt.size)
    mag = np.bincount(row, weights=mags, minlength=cnt.size)
    return sp.csr_matrix((val, indices, indptr), shape=shape), mag


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_gather_reassembles_a0(form):
    n = 8
    beta, alpha = workload_coefficients(n, True, 5)
    hh = build_hierarchy(form, n, 0, beta, alpha, assembly=True)
    asm = hh.diagnostics["assembly"]
    A0 = hh.A[0]
    assert asm["coff"][-1] == asm["ccell"].size == asm["cidx"].size
    # every cell adds s*s entries
    assert asm["ccell"].size == 6 * n ** 3 * asm["s"] ** 2
    R, mag = _gather(asm, beta, alpha, A0.shape, A0.indptr, A0.indices)
    err = np.abs(R.data - A0.data)
    cnt = np.diff(asm["coff"])
    assert np.all(err <= 4 * (cnt + 1) * EPS * mag)


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_new_coefficients_give_the_generators_hierarchy(form):
    n = 16
    b1, a1 = workload_coefficients(n, True, 5)
    b2 = block_coefficients(n, 4, -2.0, 2.0, 17)
    a2 = block_coefficients(n, 8, -1.0, 1.0, 19)
    h1 = build_hierarchy(form, n, 0, b1, a1, assembly=True)
    h2 = build_hierarchy(form, n, 0, b2, a2)
    asm = h1.diagnostics["assembly"]
    A0 = h1.A[0]
    R, mag = _gather(asm, b2, a2, A0.shape, A0.indptr, A0.indices)
    ref = h2.A[0]
    assert np.array_equal(ref.indptr, A0.indptr) and np.array_equal(ref.indices, A0.indices)
    cnt = np.diff(asm["coff"])
    assert np.all(np.abs(R.data - ref.data) <= 4 * (cnt + 1) * EPS * mag)
    A = R
    for l in range(h1.num_levels - 1):
        P1, P2 = h1.P[l].to_scipy(), h2.P[l].to_scipy()
        assert (P1 != P2).nnz == 0 and (h1.G[l].to_scipy() != h2.G[l].to_scipy()).nnz == 0
        A = (P1.T @ A @ P1).tocsr()
        An = h2.A[l + 1].to_scipy()
        assert abs(A - An).max() <= 1e-13 * abs(An).max()
