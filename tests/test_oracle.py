"""Pins of the FP64 oracle against what the paper and the mathematics fix.

  * l1-Jacobi (Section 4.1): M - A is positive semi-definite, so the eigenvalues of
    M^{-1} A lie in (0, 1]; the same holds for the auxiliary matrix G^T A G.
  * Algorithm 4.1 with the transposed post-smoother gives a symmetric positive
    definite preconditioner B (x^T B y = y^T B x), and since every factor of the
    error propagation is A-nonexpansive with an exact coarse solve, eig(B A) lies
    in (0, 1].
  * The error propagation of one V-cycle equals the product the paper states for
    the hybrid smoother (Section 4.1) around the exact two-grid correction.
  * A one-level hierarchy makes B = A^{-1}; PCG then stops after one iteration.
  * PCG reaches the dense direct solution (LAPACK through numpy) within the
    tolerance bound.
Planted mistakes (in the oracle, on the CPU) show that the pins catch them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from conftest import hierarchy, oracle_hierarchy
from oracle import OracleHierarchy, l1_row_sums, pcg
from paper_2107_05613_gb300.inputs import rhs_vector


def _dense_B(o):
    n = o.A[0].shape[0]
    return np.column_stack([o.apply(e) for e in np.eye(n)])


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_l1_smoothers_are_contractive(form):
    o = oracle_hierarchy(form, 4, 2, True)
    A = o.A[0].toarray()
    ev = sla.eigh(A, np.diag(o.m[0]), eigvals_only=True)
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12
    Aa = o.A_aux[0].toarray()
    ev = sla.eigh(Aa, np.diag(o.m_aux[0]), eigvals_only=True)
    assert ev.min() >= -1e-12 and ev.max() <= 1 + 1e-12


@pytest.mark.parametrize("form,n,L", [("hcurl", 4, 2), ("hcurl", 4, 3), ("hdiv", 4, 3), ("hcurl", 2, 2)])
def test_vcycle_spd_and_spectrum(form, n, L):
    o = oracle_hierarchy(form, n, L, True)
    B = _dense_B(o)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    A = o.A[0].toarray()
    ev = np.linalg.eigvals(B @ A)
    assert np.abs(ev.imag).max() <= 1e-10
    assert ev.real.min() > 0 and ev.real.max() <= 1 + 1e-10
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_vcycle_bilinear_symmetry_random(form):
    o = oracle_hierarchy(form, 8, 3, True)
    n = o.A[0].shape[0]
    x, y = rhs_vector(1, n), rhs_vector(2, n)
    Bx, By = o.apply(x), o.apply(y)
    assert abs(x @ By - y @ Bx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(By)
    assert x @ Bx > 0


def test_two_grid_error_propagation_matches_product_form():
    """I - B A = S^T (I - P A_c^{-1} P^T A) S, S = (I - G M_a^{-1} G^T A)(I - M^{-1} A)."""
    o = oracle_hierarchy("hcurl", 4, 2, True)
    A = o.A[0].toarray()
    n = A.shape[0]
    I = np.eye(n)
    G, P = o.G[0].toarray(), o.P[0].toarray()
    Minv = np.diag(1.0 / o.m[0])
    Mainv = np.diag(1.0 / o.m_aux[0])
    S_point = I - Minv @ A
    S_aux = I - G @ Mainv @ G.T @ A
    Ac = P.T @ A @ P
    C = I - P @ np.linalg.solve(Ac, P.T @ A)
    E_formula = S_point @ S_aux @ C @ S_aux @ S_point
    E_alg = I - _dense_B(o) @ A
    assert np.abs(E_alg - E_formula).max() <= 1e-11


def test_one_level_is_exact_solve():
    h = hierarchy("hcurl", 2, 1)
    o = OracleHierarchy.from_hierarchy(h)
    A = o.A[0].toarray()
    b = rhs_vector(3, A.shape[0])
    assert np.allclose(o.apply(b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    x, it, rr, ok = pcg(o, b)
    assert ok and it == 1 and rr <= 1e-12


@pytest.mark.parametrize("form,n,L", [("hcurl", 2, 2), ("hcurl", 4, 3), ("hdiv", 4, 2), ("hcurl", 8, 2), ("hdiv", 8, 3)])
def test_pcg_matches_dense_direct_solve(form, n, L):
    o = oracle_hierarchy(form, n, L, True)
    A = o.A[0].toarray()
    b = rhs_vector(7, A.shape[0])
    x, it, rr, ok = pcg(o, b, rtol=1e-8)
    assert ok and rr <= 1e-8
    xd = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) <= cond * 1e-8 * np.linalg.norm(xd)


def test_pcg_zero_rhs_and_maxit():
    o = oracle_hierarchy("hcurl", 4, 2, False)
    x, it, rr, ok = pcg(o, np.zeros(o.A[0].shape[0]))
    assert it == 0 and ok and not x.any()
    b = rhs_vector(3, o.A[0].shape[0])
    x, it, rr, ok = pcg(o, b, rtol=1e-14, maxit=3)
    assert it == 3 and not ok and rr > 1e-14


def test_multi_rhs_vcycle_is_columnwise():
    o = oracle_hierarchy("hdiv", 8, 2, True)
    n = o.A[0].shape[0]
    B = rhs_vector(5, n, 3)
    Z = o.apply(B)
    for j in range(3):
        assert np.allclose(Z[:, j], o.apply(B[:, j]), rtol=1e-14, atol=1e-15)


def test_iteration_counts_grow_mildly():
    """Trend of Table 5.1: bounded growth with refinement (not a value pin)."""
    its = []
    for n in (8, 16):
        o = oracle_hierarchy("hcurl", n, 2, True)
        b = rhs_vector(11, o.A[0].shape[0])
        its.append(pcg(o, b)[1])
    assert its[1] <= 2 * its[0]


# ---------------------------------------------------------------- planted mistakes
class _SameOrderPost(OracleHierarchy):
    def hybrid_transposed(self, l, x, b):      # mistake: post-smoother not transposed
        return self.hybrid(l, x, b)


class _PlainJacobi(OracleHierarchy):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.m = [self.A[l].diagonal() for l in range(self.L - 1)]   # mistake: not l1


class _ResidualSign(OracleHierarchy):
    def _point(self, l, x, b):                  # mistake: wrong residual sign
        return x + (b + self.A[l] @ x) / self.m[l]


def _planted(cls):
    h = hierarchy("hcurl", 4, 2, True)
    return cls([a.to_scipy() for a in h.A], [p.to_scipy() for p in h.P], [g.to_scipy() for g in h.G])


def test_planted_untransposed_post_smoother_breaks_symmetry():
    B = _dense_B(_planted(_SameOrderPost))
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


def test_planted_plain_jacobi_breaks_contraction():
    o = _planted(_PlainJacobi)
    ev = sla.eigh(o.A[0].toarray(), np.diag(o.m[0]), eigvals_only=True)
    assert ev.max() > 1.0 + 1e-6


def test_planted_residual_sign_breaks_spectrum():
    o = _planted(_ResidualSign)
    ev = np.linalg.eigvals(_dense_B(o) @ o.A[0].toarray()).real
    assert ev.min() <= 0 or ev.max() > 1 + 1e-6


def test_l1_row_sums_definition():
    import scipy.sparse as sp

    A = sp.csr_matrix(np.array([[4.0, -1.0, 0.0], [-1.0, 4.0, -2.0], [0.0, -2.0, 5.0]]))
    assert np.array_equal(l1_row_sums(A), [5.0, 7.0, 7.0])
