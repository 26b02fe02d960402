"""Polynomial approximation targets (Section 3.3.1) and D-free bubbles (Section 3.3.3)
in the host generator (CPU only).

With `targets=True` the generator takes the interpolants of the vector monomials up to
degree one (the constant fields e_i and the linear fields x_j e_i) as targets on the
last coarsening: their traces on coarse edges (H(curl)) or faces (H(div)), made
orthogonal to the PV trace and filtered, become new coarse dofs extended by eqs. 3.6 /
3.8, and their mass projections onto each coarse entity's D-free bubbles (H(curl):
gradients of interior vertex functions on coarse faces and cells; H(div): div-free
face functions in coarse cells), filtered by the projections' Gram matrix, are added
too; the coarsest matrix is then P^T A P.

The pins below come from the mathematics, not from the generator:
  * the PV spaces reproduce constant fields, and the enriched spaces every linear
    field (the next-to-lowest-order approximation property the targets are for);
  * the count of kept functions is the dimension the calculus predicts (H(curl): a
    linear field's tangential trace varies linearly along a straight coarse edge, and
    its surface / volume divergence spans one constant per face and per cell; H(div):
    its normal trace on a planar coarse face spans two directions beyond the PV one,
    and its curl three constants per cell);
  * the kept functions are D-free and mass-orthonormal, so with alpha = 1 their block
    of the coarsest Galerkin matrix is the identity whatever beta is, and the local
    extensions (mass-orthogonal to D-free bubbles) leave them decoupled from the rest;
  * the enrichment only appends columns, and it speeds up the H(div) two-level method.
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2107_05613_gb300.inputs import build_hierarchy, rhs_vector, workload_coefficients

CASES = [("hcurl", 8, 2), ("hcurl", 16, 3), ("hdiv", 8, 2), ("hdiv", 16, 3)]
KF = {"hcurl": 1, "hdiv": 2}


@functools.lru_cache(maxsize=None)
def _h(form, n, L, targets=False, all_spaces=False, contrast=True):
    beta, alpha = workload_coefficients(n, contrast, 11)
    return build_hierarchy(form, n, L, beta, alpha, all_spaces=all_spaces, targets=targets)


def _field_interpolant(form, n, L, field):
    """A vector field's target at the last coarsening's finer level: its interpolant on
    the finest level (the all-spaces hierarchy's interpolation of vector H1, column
    3 v + c, exact on linear fields and pinned so elsewhere), carried up by the
    co-chain projectors Pi (the integral functionals over coarse entities)."""
    k = KF[form]
    h = _h(form, n, L, all_spaces=True)
    ph = h.pihat[0][k].to_scipy()
    nv = (n + 1) ** 3
    v = np.arange(nv)
    xyz = np.stack([v // ((n + 1) ** 2), (v // (n + 1)) % (n + 1), v % (n + 1)], 1) / n
    vals = np.zeros(3 * nv)
    for c in range(3):
        vals[c::3] = field(xyz)[:, c]
    t = ph @ vals
    for l in range(L - 2):
        t = h.Pi[l][k].to_scipy() @ t
    return t


def _lsq_residual(P, t):
    y = spla.lsqr(P, t, atol=1e-15, btol=1e-15, iter_lim=50000)[0]
    return np.linalg.norm(P @ y - t) / np.linalg.norm(t)


@pytest.mark.parametrize("form,n,L", CASES)
def test_pv_spaces_reproduce_constants_and_enriched_ones_linear_fields(form, n, L):
    """Every constant field's target lies in the range of the PV-only prolongator; every
    linear field x_j e_i's lies in the range of the enriched one (measured residuals
    <= 1.4e-14), while some linear field's does not lie in the PV-only range (x e_x for
    H(curl): 0.1; y e_x for H(div): 0.1)."""
    P0 = _h(form, n, L).P[-1].to_scipy()
    P1 = _h(form, n, L, targets=True).P[-1].to_scipy()
    for c in range(3):
        t = _field_interpolant(form, n, L, lambda x, c=c: np.eye(3)[c][None, :].repeat(len(x), 0))
        assert _lsq_residual(P0, t) <= 1e-10
    for c in range(3):
        for j in range(3):
            f = lambda x, c=c, j=j: np.eye(3)[c][None, :] * x[:, j : j + 1]
            assert _lsq_residual(P1, _field_interpolant(form, n, L, f)) <= 1e-10, (c, j)
    j = 0 if form == "hcurl" else 1
    lin = _field_interpolant(form, n, L, lambda x: np.eye(3)[0][None, :] * x[:, j : j + 1])
    assert _lsq_residual(P0, lin) >= 1e-3


@pytest.mark.parametrize("form,n,L", CASES)
def test_enrichment_appends_the_predicted_number_of_functions(form, n, L):
    h, h0 = _h(form, n, L, targets=True), _h(form, n, L)
    V, E, F, T = h.counts[-1]
    P, P0 = h.P[-1].to_scipy(), h0.P[-1].to_scipy()
    added = P.shape[1] - P0.shape[1]
    assert h.diagnostics["target_functions"] == added
    if form == "hcurl":
        assert added == E + F + T        # one edge trace per coarse edge, one gradient bubble per face and cell
    elif L == 2:
        assert added == 2 * F + 5 * T    # two face traces; the curls (3) and two interpolation-error modes
    else:
        assert added == 2 * F + 3 * T    # two face traces; the curls of the linear fields
    # the PV-based columns are untouched
    assert (P[:, : P0.shape[1]] != P0).nnz == 0
    assert h.A[-1].shape == (P.shape[1], P.shape[1])


@pytest.mark.parametrize("form,n,L", CASES)
def test_bubbles_are_d_free_and_mass_orthonormal(form, n, L):
    """The cell bubbles have zero derivative (curl for H(curl), divergence for H(div))
    on the finer level, and -- D-free, with alpha = 1 -- P_b^T A P_b = I for any beta."""
    h, h0 = _h(form, n, L, targets=True), _h(form, n, L)
    V, E, F, T = h.counts[-1]
    P = h.P[-1].to_scipy()
    nc0 = h0.P[-1].shape[1]
    cells = slice(P.shape[1] - (T if form == "hcurl" else P.shape[1] - nc0 - 2 * F), P.shape[1])
    Pb = P[:, cells]
    D = h.D_all[L - 2][KF[form]].to_scipy()          # curl (faces x edges) or div (cells x faces)
    assert abs(D @ Pb).max() <= 1e-10 * abs(Pb).max()
    Af = h.A[L - 2].to_scipy()
    G = (Pb.T @ Af @ Pb).toarray()
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-9
    # and the coarsest matrix is the (symmetric) Galerkin product with the enlarged P
    Ac = h.A[-1].to_scipy().tocsr()
    ref = (P.T @ Af @ P).tocsr()
    assert abs(Ac - ref).max() <= 1e-12 * abs(ref).max()
    assert abs(Ac - Ac.T).max() == 0.0
    # the extensions of eqs. 3.6 / 3.8 satisfy phi + D* chi = 0 inside the cell, so
    # every other coarse function is mass-orthogonal to the cell's D-free bubbles: with
    # alpha = 1 the bubbles decouple from the rest of the coarsest matrix (measured
    # <= 9e-15 of its largest entry)
    nb = Pb.shape[1]
    B = Ac[Ac.shape[0] - nb:, : Ac.shape[0] - nb]
    assert B.nnz == 0 or abs(B).max() <= 1e-12 * abs(Ac).max()


@pytest.mark.parametrize("contrast", [True, False])
def test_targets_speed_up_the_hdiv_two_level_method(contrast):
    """A richer coarse space (Section 3.3.1's purpose): the H(div) two-level PCG needs
    fewer iterations with the enriched coarse space (measured on 8^3: 33 -> 25 with
    the contrast; 16^3: 37 -> 29 with and without)."""
    from oracle import OracleHierarchy, pcg

    its = []
    for tg in (False, True):
        h = _h("hdiv", 8, 2, targets=tg, contrast=contrast)
        o = OracleHierarchy.from_hierarchy(h)
        b = rhs_vector(3, h.A[0].shape[0])
        x, it, rel, _ = pcg(o, b, rtol=1e-8)
        assert rel <= 1e-8
        its.append(it)
    assert its[1] <= 0.9 * its[0], its


def test_target_options_rejected_together():
    with pytest.raises(RuntimeError):
        build_hierarchy("hdiv", 8, 2, targets=True, all_spaces=True)


@pytest.mark.parametrize("form,L", [("hcurl", 2), ("hdiv", 2), ("hcurl", 3), ("hdiv", 3)])
def test_fp32_vcycle_emulation_on_enriched_hierarchies(form, L):
    """The CPU emulation of the CUDA FP32 V-cycle (residuals of corrected iterates in
    double-float arithmetic) stays as close to the FP64 oracle's cycle on the enriched
    hierarchies as on the PV-only ones (measured energy-norm distance <= 7.7e-6 at
    16^3 with the 1e6 contrast)."""
    from fp32_emulation import EmulatedVcycle, energy_error, policy_df
    from oracle import OracleHierarchy

    h = _h(form, 16, L, targets=True)
    o = OracleHierarchy.from_hierarchy(h)
    r = rhs_vector(19, h.A[0].shape[0])
    err = energy_error(o.A[0], EmulatedVcycle(h, policy_df).apply(r), o.apply(r))
    assert err <= 1e-4, err


def _fine_fluxes(form_h, n, field):
    """The Raviart-Thomas interpolant of a vector field on the finest level: its flux
    through each face (vertices a < b < c, normal (x_b - x_a) x (x_c - x_a) / 2), by
    the three-point rule at barycentric (2/3, 1/6, 1/6) and permutations, exact for
    quadratic fields (a different rule from the generator's edge-midpoint one)."""
    F = form_h.D_all[0][1].to_scipy().tocsr()         # faces x edges
    E = form_h.D_all[0][0].to_scipy().tocsr()         # edges x vertices
    FV = (abs(F) @ abs(E)).tocsr()
    FV.sort_indices()
    vv = FV.indices.reshape(-1, 3)
    nv = (n + 1) ** 3
    v = np.arange(nv)
    X = np.stack([v // ((n + 1) ** 2), (v // (n + 1)) % (n + 1), v % (n + 1)], 1) / n
    a, b, c = X[vv[:, 0]], X[vv[:, 1]], X[vv[:, 2]]
    nr = np.cross(b - a, c - a) / 2
    flux = np.zeros(len(vv))
    for w in ((2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3)):
        p = w[0] * a + w[1] * b + w[2] * c
        flux += np.einsum("ij,ij->i", field(p), nr) / 3
    return flux


@pytest.mark.parametrize("n,L", [(8, 2), (16, 3)])
def test_degree_two_hdiv_targets_reproduce_quadratic_fields(n, L):
    """With the degree-two targets (face traces, the cross-space bubbles of eq. 3.7 and
    the D-free bubbles) the H(div) coarsest space reproduces every quadratic field's
    target (the fine interpolant carried up by the co-chain projectors): measured
    residuals <= 2.5e-14, while the degree-one space leaves about 1e-2."""
    h2 = _h("hdiv", n, L, targets=2)
    h1 = _h("hdiv", n, L, targets=True)
    ha = _h("hdiv", n, L, all_spaces=True)
    P2, P1 = h2.P[-1].to_scipy(), h1.P[-1].to_scipy()
    assert P2.shape[1] > P1.shape[1] and h2.A[-1].shape == (P2.shape[1],) * 2

    def target(field):
        t = _fine_fluxes(ha, n, field)
        for l in range(L - 2):
            t = ha.Pi[l][2].to_scipy() @ t
        return t

    for c in range(3):
        for j in range(3):
            for m in range(j, 3):
                f = lambda p, c=c, j=j, m=m: np.eye(3)[c][None, :] * (p[:, j] * p[:, m])[:, None]
                assert _lsq_residual(P2, target(f)) <= 1e-10, (c, j, m)
    quad = target(lambda p: np.eye(3)[0][None, :] * (p[:, 0] ** 2)[:, None])
    assert _lsq_residual(P1, quad) >= 1e-3
    # the fluxes of a linear field from this rule are the generator's exact ones
    lin = lambda p: np.eye(3)[1][None, :] * p[:, 2:3]
    t0 = ha.pihat[0][2].to_scipy()
    vals = np.zeros(t0.shape[1])
    nv = (n + 1) ** 3
    vtx = np.arange(nv)
    X = np.stack([vtx // ((n + 1) ** 2), (vtx // (n + 1)) % (n + 1), vtx % (n + 1)], 1) / n
    vals[1::3] = X[:, 2]
    assert np.abs(_fine_fluxes(ha, n, lin) - t0 @ vals).max() <= 1e-15


def test_degree_two_targets_speed_up_the_hdiv_two_level_method():
    """Measured on 8^3: 33 (PV only) -> 25 (degree one) -> 20 (degree two) iterations
    (16^3: 37 -> 29 -> 22)."""
    from oracle import OracleHierarchy, pcg

    its = []
    for d in (1, 2):
        h = _h("hdiv", 8, 2, targets=d)
        o = OracleHierarchy.from_hierarchy(h)
        x, it, rel, _ = pcg(o, rhs_vector(3, h.A[0].shape[0]), rtol=1e-8)
        assert rel <= 1e-8
        its.append(it)
    assert its[1] < its[0], its


def _fine_edge_integrals(form_h, n, field):
    """The Nedelec interpolant of a vector field on the finest level: the integral of
    its tangential component along each edge (a < b, tangent x_b - x_a), by the
    two-point Gauss rule, exact for cubics (a different rule from the generator's
    Simpson one)."""
    E = form_h.D_all[0][0].to_scipy().tocsr()         # edges x vertices
    E.sort_indices()
    vv = E.indices.reshape(-1, 2)
    nv = (n + 1) ** 3
    v = np.arange(nv)
    X = np.stack([v // ((n + 1) ** 2), (v // (n + 1)) % (n + 1), v % (n + 1)], 1) / n
    a, b = X[vv[:, 0]], X[vv[:, 1]]
    t = b - a
    g = 0.5 / np.sqrt(3.0)
    return sum(0.5 * np.einsum("ij,ij->i", field(a + s_ * t), t) for s_ in (0.5 - g, 0.5 + g))


@pytest.mark.parametrize("n,L", [(8, 2), (16, 3)])
def test_degree_two_hcurl_targets_reproduce_quadratic_fields(n, L):
    """With the degree-two targets (edge traces, face gradient and eq. 3.7 bubbles, the
    eq. 3.8 extensions with the curl traces' face-space extensions as targets, eq. 3.9
    and gradient cell bubbles) the H(curl) coarsest space reproduces every quadratic
    field's target: measured residuals <= 4.3e-14, the degree-one space ~1e-2."""
    h2 = _h("hcurl", n, L, targets=2)
    h1 = _h("hcurl", n, L, targets=True)
    ha = _h("hcurl", n, L, all_spaces=True)
    P2, P1 = h2.P[-1].to_scipy(), h1.P[-1].to_scipy()

    def target(field):
        t = _fine_edge_integrals(ha, n, field)
        for l in range(L - 2):
            t = ha.Pi[l][1].to_scipy() @ t
        return t

    for c in range(3):
        for j in range(3):
            for m in range(j, 3):
                f = lambda p, c=c, j=j, m=m: np.eye(3)[c][None, :] * (p[:, j] * p[:, m])[:, None]
                assert _lsq_residual(P2, target(f)) <= 1e-10, (c, j, m)
    quad = target(lambda p: np.eye(3)[0][None, :] * (p[:, 1] ** 2)[:, None])
    assert _lsq_residual(P1, quad) >= 1e-3
    # the integrals of a linear field from this rule are the generator's exact ones
    t0 = ha.pihat[0][1].to_scipy()
    vals = np.zeros(t0.shape[1])
    nv = (n + 1) ** 3
    vtx = np.arange(nv)
    vals[0::3] = (vtx % (n + 1)) / n                  # the field z e_x
    lin = _fine_edge_integrals(ha, n, lambda p: np.eye(3)[0][None, :] * p[:, 2:3])
    assert np.abs(lin - t0 @ vals).max() <= 1e-15


def test_degree_two_targets_speed_up_the_hcurl_two_level_method():
    """Degree one adds gradients, which the auxiliary-space smoother already handles
    (8^3: 33 -> 33 iterations); degree two's cross-space bubbles carry curl: 33 -> 22
    (16^3: 37 -> 36 -> 24)."""
    from oracle import OracleHierarchy, pcg

    its = []
    for d in (1, 2):
        h = _h("hcurl", 8, 2, targets=d)
        o = OracleHierarchy.from_hierarchy(h)
        x, it, rel, _ = pcg(o, rhs_vector(3, h.A[0].shape[0]), rtol=1e-8)
        assert rel <= 1e-8
        its.append(it)
    assert its[1] <= 0.8 * its[0], its


def test_target_degree_out_of_range():
    with pytest.raises(ValueError):
        build_hierarchy("hcurl", 8, 2, targets=3)
