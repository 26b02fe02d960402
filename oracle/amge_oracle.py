"""Plain FP64 oracle: hybrid-smoothed AMGe V-cycle and PCG.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every step follows the
paper in its own order; library primitives (sparse matrix-vector products, a
dense Cholesky factorisation) serve as single steps, with no fusion or reordering.

  * Algorithm 4.1 (Section 4): the V-cycle -- pre-relax, restrict the residual with
    P^T, recurse (or solve on the coarsest level), prolong with P, post-relax with
    the transposed smoother.  Called with x0 = 0 as the PCG preconditioner.
  * Eq. 4.1 (Section 4.1): one hybrid smoothing step = a point sweep on A_l, then a
    point sweep on the auxiliary matrix G^T A_l G reached through the exterior
    derivative G (D_0 for H(curl), D_1 for H(div)), corrected back through G.  The
    transposed step runs the two sweeps in the reverse order.
  * Point smoother: l1-Jacobi, M = diag(sum_j |a_ij|) (the l1-scaled point variant
    the paper cites in Section 4.1; this build's default), or the smoother of the
    paper's runs (Section 5.1): symmetric Gauss-Seidel, two sweeps for the primary
    and for the auxiliary smoothing, here in a multicolour ordering (rows sorted by
    the colour of a greedy colouring of the matrix graph, then by index).  The l1
    term of the paper's l1-scaled block variant adds, to a row's diagonal, its
    couplings to rows outside the row's processor block; with the whole matrix as
    one block it is zero, and the smoother is plain symmetric Gauss-Seidel.
  * Coarsest level: dense FP64 Cholesky solve (the default), or the paper's solver
    (Sections 4.2 and 5.1): a fixed number of PCG iterations preconditioned by the
    additive auxiliary-space preconditioner of eq. 4.2 (AuxSpaceCoarseSolver).
  * PCG (Sections 4 and 5.1): preconditioned conjugate gradients with x0 = 0 and
    one V-cycle per iteration; stop on the true FP64 relative residual
    ||b - A x|| / ||b|| <= rtol (residual replaced by the true one when the
    recursive residual first meets the tolerance).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def l1_row_sums(A) -> np.ndarray:
    """m_i = sum_j |a_ij|: the l1-Jacobi diagonal (Section 4.1 point smoother)."""
    return np.asarray(abs(A).sum(axis=1)).ravel()


def greedy_colours(S) -> np.ndarray:
    """Colour of every row of the symmetric sparsity pattern S (its nonzero entries):
    rows in index order, each taking the smallest colour no already-coloured
    neighbour has."""
    S = sp.csr_matrix(S)
    S.eliminate_zeros()
    n = S.shape[0]
    colour = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        used = {int(colour[j]) for j in S.indices[S.indptr[i]:S.indptr[i + 1]] if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def colour_order(S) -> np.ndarray:
    """The multicolour ordering: rows sorted by colour, then by index."""
    colour = greedy_colours(S)
    return np.lexsort((np.arange(colour.size), colour))


class SymmetricGaussSeidel:
    """Symmetric Gauss-Seidel for M x = b in a given row ordering: one step is a
    forward sweep (rows in order, each x_i <- x_i + (b_i - M_i x) / m_ii with the
    rows before it already updated) then a backward sweep (reverse order).  Written
    with the ordering's triangular parts: forward x <- x + (D + L)^{-1} (b - M x),
    backward x <- x + (D + U)^{-1} (b - M x), L / U the couplings to rows earlier /
    later in the ordering."""

    def __init__(self, M, order):
        M = sp.csr_matrix(M)
        self.M = M
        self.order = np.asarray(order)
        Mp = M[self.order][:, self.order].tocsr()
        self.lower = sp.tril(Mp, format="csr")
        self.upper = sp.triu(Mp, format="csr")

    def _solve(self, T, v, lower):
        return spla.spsolve_triangular(T, v, lower=lower)

    def step(self, x, b):
        o = self.order
        r = (b - self.M @ x)[o]
        x = x.copy()
        x[o] += self._solve(self.lower, r, True)           # forward sweep
        r = (b - self.M @ x)[o]
        x[o] += self._solve(self.upper, r, False)          # backward sweep
        return x


def coarse_interpolation(h, k: int):
    """The interpolation of vector H1 into space k (1 edges, 2 faces) at the coarsest
    level of generated hierarchy h (built with all spaces), by the recursion of
    Section 4.2 from the finest level's: pihat^{l+1} = Pi^l pihat^l (P_0^l (x) I_3),
    with Pi^l the co-chain projector of space k and P_0^l the H1 prolongator."""
    M = h.pihat[0][k].to_scipy()
    for l in range(h.num_levels - 1):
        Pv = sp.kron(h.P_all[l][0].to_scipy(), sp.eye(3), format="csr")
        M = (h.Pi[l][k].to_scipy() @ M @ Pv).tocsr()
    return M


class AuxSpaceCoarseSolver:
    """Coarsest-level solver of the paper's runs (Sections 4.2 and 5.1): `iters` PCG
    iterations (five) from x0 = 0 on A, preconditioned by the additive
    auxiliary-space preconditioner of eq. 4.2,

      B^{-1} = M^{-1} + Pihat S_v^{-1} Pihat^T + D B_D D^T,   S_v = Pihat^T A Pihat,

    with M the l1-Jacobi point smoother (Section 4.1) and D the exterior derivative
    into the problem space.  H(curl) (AMS): D = D_0, B_D = S_g^{-1}, S_g = D_0^T A D_0.
    H(div) (ADS): D = D_1 and B_D is the same construction for the curl-curl matrix
    A_c = D_1^T A D_1 with the edge interpolation Pihat_1: B_D = M_c^{-1} + Pihat_1
    S_c^{-1} Pihat_1^T, S_c = Pihat_1^T A_c Pihat_1 (A_c annihilates gradients, so its
    gradient term is void).  The auxiliary solves are exact: S^{-1} := the
    pseudo-inverse of S, because with natural boundary conditions S_g and S_c are
    singular (constants; gradients of quadratics); their right-hand sides D^T r and
    Pihat^T t have no component in those kernels, which D and Pihat map to zero again."""

    def __init__(self, A, pihat, D, pihat_inner=None, iters: int = 5):
        self.A = sp.csr_matrix(A)
        self.iters = iters
        self.m = l1_row_sums(self.A)
        self.Pv = sp.csr_matrix(pihat)
        self.D = sp.csr_matrix(D)
        self.Sv_inv = self._reg_inverse((self.Pv.T @ self.A @ self.Pv).toarray())
        if pihat_inner is None:                      # AMS: gradient term
            self.Sg_inv = self._reg_inverse((self.D.T @ self.A @ self.D).toarray())
            self.inner = None
        else:                                        # ADS: AMS of the curl-curl matrix
            Ac = (self.D.T @ self.A @ self.D).tocsr()
            Pi1 = sp.csr_matrix(pihat_inner)
            self.inner = (l1_row_sums(Ac), Pi1, self._reg_inverse((Pi1.T @ Ac @ Pi1).toarray()))

    @staticmethod
    def _reg_inverse(S):
        """The pseudo-inverse of the symmetric positive semi-definite S: its eigenvalues
        below 1e-12 of the largest (the kernel, zero up to rounding) dropped."""
        if not S.size:
            return S.copy()
        lam, V = np.linalg.eigh(S)
        keep = lam > 1e-12 * lam.max()
        return (V[:, keep] / lam[keep]) @ V[:, keep].T

    def precondition(self, r):
        """Eq. 4.2 (additive): the three terms summed."""
        z = _div(r, self.m) + self.Pv @ (self.Sv_inv @ (self.Pv.T @ r))
        t = self.D.T @ r
        if self.inner is None:
            y = self.Sg_inv @ t
        else:
            mc, Pi1, Sc_inv = self.inner
            y = _div(t, mc) + Pi1 @ (Sc_inv @ (Pi1.T @ t))
        return z + self.D @ y

    def solve(self, b):
        """`iters` PCG iterations from x0 = 0 (fixed count, no tolerance)."""
        x = np.zeros_like(b)
        r = b.copy()
        z = self.precondition(r)
        p = z.copy()
        rho = r @ z
        for it in range(self.iters):
            q = self.A @ p
            pq = p @ q
            if pq == 0.0:
                break
            alpha = rho / pq
            x = x + alpha * p
            r = r - alpha * q
            if it + 1 == self.iters:
                break
            z = self.precondition(r)
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
        return x


class OracleHierarchy:
    """The solve-phase operators of an AMGe hierarchy, in scipy FP64.

    A: list of level matrices (level 0 finest); P[l]: level l+1 -> level l;
    G[l]: exterior derivative into the problem space at level l (aux transition).
    """

    def __init__(self, A, P, G, nu_pre: int = 1, nu_post: int = 1, smoother: str = "l1jacobi",
                 sweeps: int = 2, gs_levels: int = None, coarse_aux: AuxSpaceCoarseSolver = None):
        self.A = [sp.csr_matrix(a, dtype=np.float64) for a in A]
        self.P = [sp.csr_matrix(p, dtype=np.float64) for p in P]
        self.G = [sp.csr_matrix(g, dtype=np.float64) for g in G]
        self.L = len(self.A)
        self.nu_pre, self.nu_post = nu_pre, nu_post
        # smoother data of every smoothing level (all but the coarsest)
        self.m = [l1_row_sums(self.A[l]) for l in range(self.L - 1)]
        self.A_aux = [(self.G[l].T @ self.A[l] @ self.G[l]).tocsr() for l in range(self.L - 1)]
        self.m_aux = [l1_row_sums(self.A_aux[l]) for l in range(self.L - 1)]
        self.smoother = smoother
        self.sweeps = sweeps
        # Gauss-Seidel on the gs_levels finest smoothing levels (all by default),
        # l1-Jacobi on the coarser ones
        self.gs_levels = (self.L - 1) if gs_levels is None else min(gs_levels, self.L - 1)
        if smoother == "gs":
            # orderings from the sparsity patterns (the aux pattern symbolic: entries
            # that cancel numerically still couple)
            self.gs = []
            self.gs_aux = []
            for l in range(self.gs_levels):
                pa = abs(self.A[l])
                pg = abs(self.G[l])
                self.gs.append(SymmetricGaussSeidel(self.A[l], colour_order(pa)))
                self.gs_aux.append(SymmetricGaussSeidel(self.A_aux[l], colour_order((pg.T @ pa @ pg).tocsr())))
        elif smoother != "l1jacobi":
            raise ValueError("smoother must be 'l1jacobi' or 'gs'")
        # coarsest level: dense Cholesky factor, or the auxiliary-space solver
        Ac = self.A[-1].toarray()
        self.coarse_factor = sla.cho_factor(Ac, lower=True)
        self.coarse_aux = coarse_aux

    @classmethod
    def from_blob(cls, blob: bytes):
        """Read a serialized hierarchy: a 32-byte header ("AMGEBLOB", version 1, form,
        levels L, nu_pre, nu_post, 0), then A_0..A_{L-1}, P_0..P_{L-2}, G_0..G_{L-2},
        each as int32 rows, int32 cols, int64 nnz, int32 row_ptr, int32 col, float64
        values; little-endian, sections padded to multiples of 8 bytes."""
        buf = memoryview(blob)
        if bytes(buf[:8]) != b"AMGEBLOB" or np.frombuffer(buf[8:12], "<u4")[0] != 1:
            raise ValueError("not a version-1 hierarchy blob")
        form, L, nu_pre, nu_post, _ = (int(v) for v in np.frombuffer(buf[12:32], "<i4"))
        off = 32
        mats = []
        for _ in range(3 * L - 2):
            nr, nc = (int(v) for v in np.frombuffer(buf[off:off + 8], "<i4"))
            nnz = int(np.frombuffer(buf[off + 8:off + 16], "<i8")[0])
            off += 16
            rp = np.frombuffer(buf[off:off + 4 * (nr + 1)], "<i4")
            off += 4 * (nr + 1) + (-4 * (nr + 1)) % 8
            ci = np.frombuffer(buf[off:off + 4 * nnz], "<i4")
            off += 4 * nnz + (-4 * nnz) % 8
            v = np.frombuffer(buf[off:off + 8 * nnz], "<f8")
            off += 8 * nnz
            mats.append(sp.csr_matrix((v, ci, rp), shape=(nr, nc)))
        if off != len(buf):
            raise ValueError("trailing bytes after the last matrix")
        return cls(mats[:L], mats[L:2 * L - 1], mats[2 * L - 1:], nu_pre, nu_post)

    @classmethod
    def from_hierarchy(cls, h, nu_pre: int = 1, nu_post: int = 1, smoother: str = "l1jacobi", sweeps: int = 2,
                       gs_levels: int = None, coarse: str = "dense", coarse_iters: int = 5):
        """coarse: 'dense' (Cholesky) or 'aux' (AuxSpaceCoarseSolver; h built with all
        spaces)."""
        aux = None
        if coarse == "aux":
            L = h.num_levels
            A = h.A[-1].to_scipy()
            if h.form == "hcurl":
                aux = AuxSpaceCoarseSolver(A, coarse_interpolation(h, 1), h.D_all[L - 1][0].to_scipy(),
                                           iters=coarse_iters)
            else:
                aux = AuxSpaceCoarseSolver(A, coarse_interpolation(h, 2), h.D_all[L - 1][1].to_scipy(),
                                           coarse_interpolation(h, 1), iters=coarse_iters)
        elif coarse != "dense":
            raise ValueError("coarse must be 'dense' or 'aux'")
        return cls([a.to_scipy() for a in h.A], [p.to_scipy() for p in h.P],
                   [g.to_scipy() for g in h.G], nu_pre, nu_post, smoother, sweeps, gs_levels, aux)

    # ---------------------------------------------------------------- smoothers
    def _point(self, l, x, b):
        """x <- x + M^{-1} (b - A x).  l1-Jacobi: M = l1 diagonal (symmetric, so
        M^{-T} = M^{-1}); Gauss-Seidel: `sweeps` symmetric steps (symmetric as well)."""
        if self.smoother == "gs" and l < self.gs_levels:
            for _ in range(self.sweeps):
                x = self.gs[l].step(x, b)
            return x
        return x + _div(b - self.A[l] @ x, self.m[l])

    def _aux(self, l, x, b):
        """x <- x + G M_aux^{-1} G^T (b - A x) (second line of eq. 4.1); with
        Gauss-Seidel, M_aux^{-1} t is `sweeps` symmetric steps on A_aux y = t from y = 0."""
        G = self.G[l]
        t = G.T @ (b - self.A[l] @ x)
        if self.smoother == "gs" and l < self.gs_levels:
            y = np.zeros_like(t)
            for _ in range(self.sweeps):
                y = self.gs_aux[l].step(y, t)
            return x + G @ y
        return x + G @ _div(t, self.m_aux[l])

    def hybrid(self, l, x, b):
        """One step of eq. 4.1: point sweep on A_l, then the auxiliary sweep."""
        x = self._point(l, x, b)
        return self._aux(l, x, b)

    def hybrid_transposed(self, l, x, b):
        """The transposed step: the two sweeps of eq. 4.1 in reverse order."""
        x = self._aux(l, x, b)
        return self._point(l, x, b)

    # ---------------------------------------------------------------- V-cycle
    def coarse_solve(self, b):
        if self.coarse_aux is not None:
            return self.coarse_aux.solve(b)
        return sla.cho_solve(self.coarse_factor, b)

    def vcycle(self, b, l: int = 0, x0=None):
        """Algorithm 4.1 at level l: returns x = x0 + B^{-1}(b - A x0) (x0 = 0 default)."""
        if self.L == 1:
            return self.coarse_solve(b)
        x = np.zeros_like(b) if x0 is None else x0.copy()
        for _ in range(self.nu_pre):                      # pre-relax
            x = self.hybrid(l, x, b)
        r_c = self.P[l].T @ (b - self.A[l] @ x)           # restrict the residual
        if l + 1 == self.L - 1:                           # coarsest level reached
            e_c = self.coarse_solve(r_c)
        else:
            e_c = self.vcycle(r_c, l + 1)
        x = x + self.P[l] @ e_c                           # correct
        for _ in range(self.nu_post):                     # post-relax with M^{-T}
            x = self.hybrid_transposed(l, x, b)
        return x

    def apply(self, r):
        """The preconditioner B^{-1} r: one V-cycle from x0 = 0 at the finest level."""
        return self.vcycle(r, 0)


def _div(v, d):
    return v / d if v.ndim == 1 else v / d[:, None]


def pcg(h: OracleHierarchy, b, rtol: float = 1e-8, maxit: int = 1000):
    """PCG with one V-cycle per iteration, x0 = 0 (Section 4, Section 5.1).

    Returns (x, iterations, true relative residual, converged).  The iteration count
    is the number of products A p.
    """
    A = h.A[0]
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    r = b.copy()
    z = h.apply(r)
    p = z.copy()
    rho = r @ z
    it = 0
    converged = False
    while it < maxit:
        q = A @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if np.linalg.norm(r) <= rtol * bnorm:
            r_true = b - A @ x
            if np.linalg.norm(r_true) <= rtol * bnorm:
                converged = True
                break
            r = r_true
        z = h.apply(r)
        rho_new = r @ z
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    relres = np.linalg.norm(b - A @ x) / bnorm
    return x, it, relres, converged
