"""Pins of the oracle's Gauss-Seidel smoother (the smoother of the paper's runs,
Section 5.1: symmetric Gauss-Seidel, two sweeps for the primary and the auxiliary
smoothing of the hybrid smoother, eq. 4.1), against what the definition and the
mathematics fix:

  * the greedy colouring is a proper colouring (no coupling inside a colour), so
    Gauss-Seidel in the colour-sorted order updates a whole colour independently;
  * one symmetric step equals the definition written as a row-by-row loop (forward
    over the ordering, then backward), each row seeing the rows already updated;
  * for SPD A the symmetric Gauss-Seidel preconditioner M satisfies
    eig(M^{-1} A) in (0, 1] (the error propagation is A-nonexpansive);
  * the V-cycle with it is symmetric positive definite with eig(B A) in (0, 1];
  * PCG with it reaches the dense direct solution within the tolerance bound;
  * a planted mistake (the forward sweep only, a non-symmetric smoother) breaks the
    symmetry pin.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from conftest import hierarchy
from oracle import OracleHierarchy, SymmetricGaussSeidel, colour_order, greedy_colours, pcg
from paper_2107_05613_gb300.inputs import rhs_vector


def _gs_loop(M, order, x, b):
    """One symmetric Gauss-Seidel step as the definition: rows in order, then reversed."""
    M = M.toarray()
    x = x.copy()
    for i in order:
        x[i] += (b[i] - M[i] @ x) / M[i, i]
    for i in order[::-1]:
        x[i] += (b[i] - M[i] @ x) / M[i, i]
    return x


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_colouring_is_proper(form):
    o = OracleHierarchy.from_hierarchy(hierarchy(form, 4, 2, True), smoother="gs")
    pa, pg = abs(o.A[0]), abs(o.G[0])
    # the aux pattern is the symbolic product (numeric G^T A G cancels some entries
    # to zero on one side of the diagonal only)
    for M in (o.A[0], (pg.T @ pa @ pg).tocsr(), o.A[0][:50][:, :50]):
        S = sp.csr_matrix(abs(M))
        col = greedy_colours(S)
        coo = S.tocoo()
        off = coo.row != coo.col
        assert np.all(col[coo.row[off]] != col[coo.col[off]])
        assert col.min() == 0
        # every colour up to the largest is used (greedy never skips one)
        assert set(np.unique(col)) == set(range(col.max() + 1))
    order = colour_order(abs(o.A[0]))
    assert sorted(order.tolist()) == list(range(o.A[0].shape[0]))
    c = greedy_colours(abs(o.A[0]))[order]
    assert np.all(np.diff(c) >= 0)


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_symmetric_step_is_the_row_loop(form):
    hh = hierarchy(form, 2, 2, True)
    A = hh.A[0].to_scipy().tocsr()
    rng = np.random.default_rng(3)
    for order in (colour_order(abs(A)), rng.permutation(A.shape[0])):
        g = SymmetricGaussSeidel(A, order)
        x = rng.uniform(-1, 1, A.shape[0])
        b = rng.uniform(-1, 1, A.shape[0])
        ref = _gs_loop(A, order, x, b)
        assert np.abs(g.step(x, b) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_symmetric_gs_spectrum(form):
    o = OracleHierarchy.from_hierarchy(hierarchy(form, 2, 2, True), smoother="gs")
    for M, g in ((o.A[0], o.gs[0]), (o.A_aux[0], o.gs_aux[0])):
        n = M.shape[0]
        # M_sgs^{-1}: one symmetric step from 0 applied to the unit vectors
        Minv = np.column_stack([g.step(np.zeros(n), e) for e in np.eye(n)])
        assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
        ev = np.linalg.eigvals(Minv @ M.toarray())
        assert np.abs(ev.imag).max() <= 1e-8
        # the aux matrix is singular (its kernel: the gradients of the aux space)
        lo = -1e-10 if M is o.A_aux[0] else 1e-12
        assert ev.real.min() > lo and ev.real.max() <= 1 + 1e-10


def _dense_B(o):
    n = o.A[0].shape[0]
    return np.column_stack([o.apply(e) for e in np.eye(n)])


@pytest.mark.parametrize("form,n,L,gs_levels", [("hcurl", 2, 2, None), ("hdiv", 2, 2, None), ("hcurl", 4, 3, None),
                                                 ("hdiv", 4, 3, 1)])
def test_vcycle_with_gs_is_spd_and_contractive(form, n, L, gs_levels):
    """All smoothing levels with Gauss-Seidel, or the finest only (l1-Jacobi below)."""
    o = OracleHierarchy.from_hierarchy(hierarchy(form, n, L, True), smoother="gs", gs_levels=gs_levels)
    B = _dense_B(o)
    assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()
    ev = np.linalg.eigvals(B @ o.A[0].toarray())
    assert np.abs(ev.imag).max() <= 1e-8
    assert ev.real.min() > 0 and ev.real.max() <= 1 + 1e-8


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_pcg_with_gs_reaches_dense_solution(form):
    hh = hierarchy(form, 4, 2, True)
    o = OracleHierarchy.from_hierarchy(hh, smoother="gs")
    A = o.A[0].toarray()
    b = rhs_vector(11, A.shape[0])
    x, it, rr, ok = pcg(o, b, rtol=1e-8)
    xd = np.linalg.solve(A, b)
    assert ok and rr <= 1e-8
    assert np.linalg.norm(x - xd) <= np.linalg.cond(A) * 1e-8 * np.linalg.norm(xd)
    _, it_j, _, _ = pcg(OracleHierarchy.from_hierarchy(hh), b, rtol=1e-8)
    assert it < it_j                      # the stronger smoother needs fewer iterations


def test_planted_forward_only_smoother_breaks_symmetry(monkeypatch):
    o = OracleHierarchy.from_hierarchy(hierarchy("hcurl", 2, 2, True), smoother="gs")

    def forward_only(self, x, b):
        o_ = self.order
        r = (b - self.M @ x)[o_]
        x = x.copy()
        x[o_] += sp.linalg.spsolve_triangular(self.lower, r, lower=True)
        return x

    monkeypatch.setattr(SymmetricGaussSeidel, "step", forward_only)
    B = _dense_B(o)
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()
