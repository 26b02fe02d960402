"""Pins of the auxiliary-space data and the oracle's auxiliary-space coarse solver
(Sections 3.2.2 and 4.2), against what the definitions and the mathematics fix:

  * co-chain projectors: Pi P = I (eq. 3.3) and Pi_{k+1} D_k = D_k^H Pi_k (the
    commutativity the paper requires) on every level and space, exactly;
  * the finest interpolation pihat reproduces, for linear vector fields, the edge
    integrals and face fluxes computed here from the vertex coordinates (midpoint
    and centroid rules are exact for linear fields; face orientation taken from the
    signed boundary chain in D_1, not from a vertex-order convention);
  * the commuting diagram on the finest level: pihat_1 grad(phi) = D_0 phi for linear
    phi, D_1 pihat_1 w = pihat_2 curl(w) for linear w;
  * eq. 4.2's preconditioner is symmetric positive definite, and PCG with it reaches
    the dense solution of the coarsest problem;
  * a planted mistake (the interpolation with one orientation flipped) breaks the
    exactness pin.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import AuxSpaceCoarseSolver, OracleHierarchy, coarse_interpolation, pcg
from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector
from paper_2107_05613_gb300.inputs.rng import workload_coefficients


def _hier(form, n, L, contrast=True):
    b, a = workload_coefficients(n, contrast, 11) if contrast else (None, None)
    return build_hierarchy(form, n, L, b, a, all_spaces=True)


def _coords(n):
    n1 = n + 1
    v = np.arange(n1 ** 3)
    return np.stack([v // (n1 * n1), (v // n1) % n1, v % n1], axis=1) / n


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_cochain_projectors(form):
    hh = _hier(form, 8, 3)
    for l in range(hh.num_levels - 1):
        for k in range(4):
            Pi, P = hh.Pi[l][k].to_scipy(), hh.P_all[l][k].to_scipy()
            assert abs(Pi @ P - sp.eye(P.shape[1])).max() <= 1e-14, (l, k)
        for k in range(3):
            lhs = hh.Pi[l][k + 1].to_scipy() @ hh.D_all[l][k].to_scipy()
            rhs = hh.D_all[l + 1][k].to_scipy() @ hh.Pi[l][k].to_scipy()
            assert abs(lhs - rhs).max() == 0, (l, k)


def _linear_field(rng, X):
    c = rng.uniform(-1, 1, 3)
    B = rng.uniform(-1, 1, (3, 3))
    return c, B, (c[None, :] + X @ B.T)          # r(x) = c + B x at the vertices


def _edge_geometry(hh, X):
    D0 = hh.D_all[0][0].to_scipy().tocoo()
    tail = np.zeros(D0.shape[0], int)
    head = np.zeros(D0.shape[0], int)
    tail[D0.row[D0.data < 0]] = D0.col[D0.data < 0]
    head[D0.row[D0.data > 0]] = D0.col[D0.data > 0]
    return tail, head


def _face_vector_areas(hh, X, tail, head):
    """Vector area of every face from its signed boundary chain (rows of D_1):
    (1/2) sum_e s_e (x_tail(e) x x_head(e))."""
    D1 = hh.D_all[0][1].to_scipy().tocoo()
    cr = np.cross(X[tail], X[head])
    out = np.zeros((D1.shape[0], 3))
    np.add.at(out, D1.row, 0.5 * D1.data[:, None] * cr[D1.col])
    return out


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_fine_interpolation_exact_on_linear_fields(form):
    hh = _hier(form, 4, 1, contrast=False)
    X = _coords(4)
    rng = np.random.default_rng(1)
    c, B, R = _linear_field(rng, X)
    r = R.ravel()                                  # column 3 v + c
    tail, head = _edge_geometry(hh, X)
    mid = 0.5 * (X[tail] + X[head])
    ref_e = np.einsum("ij,ij->i", X[head] - X[tail], c[None, :] + mid @ B.T)
    assert np.abs(hh.pihat[0][1].to_scipy() @ r - ref_e).max() <= 1e-14
    # faces: flux of r through the oriented triangle = vector area . r(centroid)
    D1 = hh.D_all[0][1].to_scipy()
    S = _face_vector_areas(hh, X, tail, head)
    fv = [np.unique(np.concatenate([tail[D1.indices[D1.indptr[f]:D1.indptr[f + 1]]],
                                    head[D1.indices[D1.indptr[f]:D1.indptr[f + 1]]]]))
          for f in range(D1.shape[0])]
    cen = np.array([X[v].mean(axis=0) for v in fv])
    ref_f = np.einsum("ij,ij->i", S, c[None, :] + cen @ B.T)
    assert np.abs(hh.pihat[0][2].to_scipy() @ r - ref_f).max() <= 1e-14


def test_commuting_diagram_on_the_finest_level():
    hh = _hier("hdiv", 4, 1, contrast=False)
    X = _coords(4)
    rng = np.random.default_rng(2)
    g = rng.uniform(-1, 1, 3)                       # phi(x) = g . x: grad phi = g
    phi = X @ g
    grad = np.tile(g, (X.shape[0], 1)).ravel()
    Pi1, Pi2 = hh.pihat[0][1].to_scipy(), hh.pihat[0][2].to_scipy()
    D0, D1 = hh.D_all[0][0].to_scipy(), hh.D_all[0][1].to_scipy()
    assert np.abs(Pi1 @ grad - D0 @ phi).max() <= 1e-14
    c, B, W = _linear_field(rng, X)                # curl(c + B x) = constant
    curl = np.array([B[2, 1] - B[1, 2], B[0, 2] - B[2, 0], B[1, 0] - B[0, 1]])
    assert np.abs(D1 @ (Pi1 @ W.ravel()) - Pi2 @ np.tile(curl, (X.shape[0], 1)).ravel()).max() <= 1e-14


def test_planted_orientation_flip_breaks_exactness():
    hh = _hier("hcurl", 4, 1, contrast=False)
    X = _coords(4)
    rng = np.random.default_rng(3)
    c, B, R = _linear_field(rng, X)
    tail, head = _edge_geometry(hh, X)
    mid = 0.5 * (X[tail] + X[head])
    ref = np.einsum("ij,ij->i", X[head] - X[tail], c[None, :] + mid @ B.T)
    M = hh.pihat[0][1].to_scipy().tolil()
    M[5, :] = -M[5, :]                              # edge 5 oriented the other way
    assert np.abs(M.tocsr() @ R.ravel() - ref).max() > 1e-3


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_aux_preconditioner_spd_and_coarse_pcg(form):
    hh = _hier(form, 8, 2)
    L = hh.num_levels
    A = hh.A[-1].to_scipy()
    if form == "hcurl":
        s = AuxSpaceCoarseSolver(A, coarse_interpolation(hh, 1), hh.D_all[L - 1][0].to_scipy())
    else:
        s = AuxSpaceCoarseSolver(A, coarse_interpolation(hh, 2), hh.D_all[L - 1][1].to_scipy(),
                                 coarse_interpolation(hh, 1))
    n = A.shape[0]
    B = np.column_stack([s.precondition(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    b = rhs_vector(4, n)
    xe = np.linalg.solve(A.toarray(), b)
    x5 = s.solve(b)
    e5 = np.sqrt((x5 - xe) @ (A @ (x5 - xe)) / (xe @ (A @ xe)))
    s.iters = 30
    x30 = s.solve(b)
    e30 = np.sqrt((x30 - xe) @ (A @ (x30 - xe)) / (xe @ (A @ xe)))
    assert e5 <= 1e-2 and e30 <= max(1e-9, 1e-3 * e5), (e5, e30)


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_vcycle_with_aux_coarse_solver(form):
    """The V-cycle with the paper's coarsest solver: PCG reaches the tolerance in the
    iteration count of the dense coarsest solve (+2)."""
    hh = _hier(form, 8, 2)
    b = rhs_vector(5, hh.A[0].shape[0])
    _, it_d, _, ok_d = pcg(OracleHierarchy.from_hierarchy(hh), b)
    x, it_a, rr, ok_a = pcg(OracleHierarchy.from_hierarchy(hh, coarse="aux"), b)
    assert ok_d and ok_a and rr <= 1e-8 and it_a <= it_d + 2, (it_a, it_d)
