"""Pins of the generated AMGe hierarchy (input data of the solve phase).

Each test checks the generator against something the paper or the mathematics
fixes: closed-form entity counts, the de Rham identities D_{k+1} D_k = 0 (eq. 2.3,
Section 2.2.1) bit-exact in integers at every level (eq. 3.2), Whitney-form
identities (stiffness = D^T (mass) D), the commuting property (eq. 3.3) in the
form D_k P_k = P_{k+1} D_k^H, Galerkin RAP (Section 3.2.1), PV rows (eq. 3.5) and
the worked prolongator column of Fig. 3.3.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from conftest import hierarchy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _int(M):
    """CSR with integer values (the incidences are exact small integers)."""
    S = M.to_scipy()
    assert np.all(S.data == np.round(S.data))
    return sp.csr_matrix((S.data.astype(np.int64), S.indices, S.indptr), shape=S.shape)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_fine_entity_counts_closed_form(n):
    h = hierarchy("hcurl", n, 1)
    V, E, F, T = h.counts[0]
    assert V == (n + 1) ** 3
    assert E == 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3   # axis + face diagonals + body diagonals
    assert F == 6 * n * n * (n + 1) + 6 * n ** 3                      # 2 per grid square + 6 inside each cube
    assert T == 6 * n ** 3
    assert V - E + F - T == 1                                          # contractible domain


@pytest.mark.parametrize("form,n,L", [("hcurl", 4, 3), ("hdiv", 8, 4), ("hcurl", 16, 2)])
def test_coarse_levels_are_hex_topologies(form, n, L):
    h = hierarchy(form, n, L)
    for l in range(1, L):
        m = n >> l
        assert h.counts[l] == ((m + 1) ** 3, 3 * m * (m + 1) ** 2, 3 * m * m * (m + 1), m ** 3)


@pytest.mark.parametrize("form,n,L", [("hcurl", 4, 3), ("hdiv", 8, 4), ("hcurl", 8, 2)])
def test_de_rham_exact_integers_every_level(form, n, L):
    """D_{k+1} D_k = 0 exactly, in integer arithmetic, at every level (eqs. 2.3, 3.2)."""
    h = hierarchy(form, n, L)
    for l in range(L):
        D = [_int(h.D_all[l][k]) for k in range(3)]
        assert (D[1] @ D[0]).count_nonzero() == 0
        assert (D[2] @ D[1]).count_nonzero() == 0
        for k in range(3):
            assert set(np.unique(D[k].data)) <= {-1, 1}


@pytest.mark.parametrize("n,L", [(1, 1), (2, 2)])
def test_exactness_ranks(n, L):
    """Exactness (eq. 2.4 / 3.2): rank D_0 = V-1, rank D_1 = E-V+1, rank D_2 = T."""
    h = hierarchy("hcurl", n, L)
    for l in range(L):
        V, E, F, T = h.counts[l]
        D = [h.D_all[l][k].to_scipy().toarray() for k in range(3)]
        assert np.linalg.matrix_rank(D[0]) == V - 1
        assert np.linalg.matrix_rank(D[1]) == E - (V - 1)
        assert np.linalg.matrix_rank(D[2]) == T


def _stiffness_and_mass(form, n):
    """Split A = beta K + alpha M using two generated hierarchies (beta = 1 and 2)."""
    from paper_2107_05613_gb300.inputs import build_hierarchy

    nt = 6 * n ** 3
    A1 = build_hierarchy(form, n, 1, beta=np.ones(nt), alpha=np.ones(nt)).A[0].to_scipy()
    A2 = build_hierarchy(form, n, 1, beta=2 * np.ones(nt), alpha=np.ones(nt)).A[0].to_scipy()
    K = (A2 - A1).tocsr()
    return K, (A1 - K).tocsr()


@pytest.mark.parametrize("n", [2, 3])
def test_whitney_div_stiffness_is_incidence_product(n):
    """(div w_f, div w_g) = (D_2^T M_L2 D_2)_{fg} with the P0 dofs of unit integral."""
    K, _ = _stiffness_and_mass("hdiv", n)
    D2 = hierarchy("hdiv", n, 1).D_all[0][2].to_scipy()
    vol_inv = 6.0 * n ** 3                      # 1 / |tet|, |tet| = h^3 / 6
    ref = (D2.T @ D2) * vol_inv
    assert abs(K - ref).max() <= 1e-12 * abs(ref).max()


@pytest.mark.parametrize("n", [2, 3])
def test_whitney_curl_stiffness_is_incidence_product(n):
    """(curl w_e, curl w_g) = (D_1^T M_RT D_1)_{eg}: curl maps Nedelec into RT exactly."""
    Kc, _ = _stiffness_and_mass("hcurl", n)
    _, MF = _stiffness_and_mass("hdiv", n)
    D1 = hierarchy("hcurl", n, 1).D_all[0][1].to_scipy()
    ref = D1.T @ MF @ D1
    assert abs(Kc - ref).max() <= 1e-12 * abs(ref).max()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_whitney_masses_reproduce_constant_fields(n):
    """A constant field c has edge dofs c.(x_b - x_a) and face dofs c.(area normal);
    its L2 energy on the unit cube is |c|^2 exactly."""
    h = hierarchy("hcurl", n, 1)
    _, ME = _stiffness_and_mass("hcurl", n)
    _, MF = _stiffness_and_mass("hdiv", n)
    n1 = n + 1
    idx = np.arange(n1 ** 3)
    X = np.stack([idx // (n1 * n1), (idx // n1) % n1, idx % n1], axis=1) / n
    c = np.array([0.3, -1.1, 0.7])
    D0 = h.D_all[0][0].to_scipy()
    xe = D0 @ (X @ c)                      # circulation of c along each edge = grad of c.x
    assert abs(xe @ (ME @ xe) - c @ c) < 1e-12
    # face dofs of c: D_1 applied to the edge dofs of a vector potential a(x) = c x x / 2
    a_at = lambda P: 0.5 * np.cross(np.broadcast_to(c, P.shape), P)
    E = D0.shape[0]
    ev = D0.indices.reshape(E, 2)
    xa = np.einsum("ij,ij->i", 0.5 * (a_at(X[ev[:, 0]]) + a_at(X[ev[:, 1]])), X[ev[:, 1]] - X[ev[:, 0]])
    xf = h.D_all[0][1].to_scipy() @ xa     # flux of curl a = c through each face (Stokes)
    assert abs(xf @ (MF @ xf) - c @ c) < 1e-12


@pytest.mark.parametrize("form,n,L", [("hcurl", 4, 3), ("hdiv", 4, 3), ("hcurl", 8, 4), ("hdiv", 8, 2)])
def test_commuting_property(form, n, L):
    """Eq. 3.3 multiplied by P_k: D_k P_k = P_{k+1} D_k^H for every space, every level."""
    h = hierarchy(form, n, L, contrast=True, all_spaces=True)
    for l in range(L - 1):
        for k in range(3):
            Pk, Pk1 = h.P_all[l][k], h.P_all[l][k + 1]
            lhs = h.D_all[l][k].to_scipy() @ Pk.to_scipy()
            rhs = Pk1.to_scipy() @ h.D_all[l + 1][k].to_scipy()
            scale = max(abs(lhs).max(), 1.0)
            assert abs(lhs - rhs).max() <= 1e-12 * scale, (l, k)


@pytest.mark.parametrize("form,n,L", [("hcurl", 8, 4), ("hdiv", 8, 4), ("hcurl", 16, 2)])
def test_galerkin_rap(form, n, L):
    """A_{l+1} = P_l^T A_l P_l (Section 3.2.1), symmetric."""
    h = hierarchy(form, n, L, contrast=True)
    for l in range(L):
        A = h.A[l].to_scipy()
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
        if l + 1 < L:
            RAP = h.P[l].to_scipy().T @ A @ h.P[l].to_scipy()
            assert abs(RAP - h.A[l + 1].to_scipy()).max() <= 1e-12 * abs(RAP).max()


def test_pv_rows_and_full_rank():
    """Fine dofs on a coarse entity carry the PV weight +-1/#constituents (eq. 3.5)."""
    h = hierarchy("hcurl", 4, 3, all_spaces=True)
    # constituents per coarse entity: level 0 (tets, triangles, fine edges), level 1 (hex pieces)
    per = {0: {0: 1, 1: 2, 2: 8, 3: 48}, 1: {0: 1, 1: 2, 2: 4, 3: 8}}
    for l in range(2):
        for k in range(4):
            P = h.P_all[l][k].to_scipy()
            single = np.diff(P.indptr) == 1
            vals = np.abs(P.data[P.indptr[:-1][single]])
            assert np.all(vals == 1.0 / per[l][k]), (l, k)
            assert np.linalg.matrix_rank(P.toarray()) == P.shape[1]


def test_fig3_3_h1_column_along_coarse_edge():
    """Fig. 3.3: the coarse H1 basis function is 1 at its vertex and 1/2 at the
    midpoint of each coarse edge of two fine segments (0 at the far end)."""
    golden = json.load(open(os.path.join(GOLDEN, "fig3_3_h1_edge_extension.json")))["values_from_vertex"]
    h = hierarchy("hcurl", 4, 2, all_spaces=True)
    P0 = h.P_all[0][0].to_scipy().toarray()      # vertices x coarse vertices
    D0 = h.D_all[0][0].to_scipy()
    n1 = 5
    # coarse vertex at fine vertex (0,0,0); coarse edge along x: fine vertices (0,0,0),(1,0,0),(2,0,0)
    vid = lambda i, j, k: (i * n1 + j) * n1 + k
    col = int(np.argmax(P0[vid(0, 0, 0)]))
    got = [P0[vid(i, 0, 0), col] for i in range(3)]
    assert got == golden
    assert D0.shape[1] == n1 ** 3


def test_local_problem_diagnostics():
    """Stokes: every eq. 3.6 multiplier equals the coarse incidence (+-1) exactly;
    every local saddle-point solve has a tiny residual."""
    h = hierarchy("hcurl", 8, 4, contrast=True, all_spaces=True)
    assert h.diagnostics["lambda_dev"] <= 1e-13
    assert h.diagnostics["local_residual"] <= 1e-12
    assert h.diagnostics["incidence_dev"] == 0.0


def test_coefficients_enter_only_the_operator():
    """Coarse spaces do not depend on beta (mass coefficient 1): P identical, A not."""
    a = hierarchy("hcurl", 16, 2, contrast=False)
    b = hierarchy("hcurl", 16, 2, contrast=True)
    assert np.array_equal(a.P[0].data, b.P[0].data)
    assert not np.allclose(a.A[0].data, b.A[0].data)


def test_rhs_and_coefficient_generators():
    from paper_2107_05613_gb300.inputs import rhs_vector, splitmix64_uniform
    from paper_2107_05613_gb300.inputs.rng import block_coefficients

    # SplitMix64 reference outputs for seed 0 (first two 64-bit outputs of the
    # published generator: 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4)
    u = splitmix64_uniform(0, 2)
    assert u[0] == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    assert u[1] == (0x6E789E6AA1B965F4 >> 11) / 2.0 ** 53
    r = rhs_vector(5, 1000)
    assert r.min() >= -1 and r.max() < 1
    beta = block_coefficients(16, 8, -3.0, 3.0, 9)
    assert beta.shape == (6 * 16 ** 3,)
    assert len(np.unique(beta)) == 8 and beta.min() >= 1e-3 and beta.max() <= 1e3
