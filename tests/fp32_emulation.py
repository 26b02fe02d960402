"""CPU emulation of the FP32 V-cycle, with the precision of each step selectable.

Test helper, not part of the product: it restates, in numpy/scipy, the order of
steps the CUDA V-cycle takes (Algorithm 4.1 with the hybrid smoother of eq. 4.1,
the residual after an aux sweep updated as r - (A G) y where the CUDA path stores
A G, the first point sweep from zero as x = m^-1 b), and runs every product either
in FP32 (float32 values, float32 sums, as scipy's float32 CSR product forms them)
or in FP64 on FP32 vectors (float64 values and sums, result rounded to float32).
The coarsest solve is FP64 (dense Cholesky), as on the GPU.

It shows on the CPU which rounding breaks the FP32 V-cycle under coefficient
contrast: the residuals b - A x of iterates that carry a correction through G or P
(the gradient / curl part of A x cancels there, and FP32 rounding of A's values or
of the sums swamps it).  Step names:
  'pre'   first residual of a level, x = m^-1 b (no correction yet)
  'pre2'  residual after the pre-smoothing aux sweep (levels without the A G form)
  'post'  residual after the coarse-grid correction x += P e
  'post2' final point sweep after the post-smoothing aux sweep (no A G form)
  'gt', 'g', 'ag', 'pt', 'p'  the other products
A policy maps (step, level) to 32 (all FP32), 64 (FP64 values and sums) or 48
(double-float: FP32 pairs for values and sums, see resid_df).  `vec`
is the vector type between steps (float32 as on the GPU; float64 with policy_fp64
makes the emulation an FP64 V-cycle, which pins its step order to the oracle).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

f32, f64 = np.float32, np.float64
EPS64 = np.finfo(f64).eps

CORRECTED = ("pre2", "post", "post2")


def policy_fp32(step, level):
    """Every product in FP32."""
    return 32


def policy_wide(step, level):
    """The CUDA FP32 V-cycle: residuals of corrected iterates on the FP64 operator."""
    return 64 if step in CORRECTED else 32


def policy_fp64(step, level):
    return 64


def policy_df(step, level):
    """Residuals of corrected iterates in double-float arithmetic (below), the rest FP32."""
    return 48 if step in CORRECTED else 32


def split_df(v):
    """A value as the float32 pair hi + lo (hi = fl32(v), lo = fl32(v - hi))."""
    hi = v.astype(f32)
    lo = (v - hi.astype(f64)).astype(f32)
    return hi, lo


def resid_df(A, x, b):
    """b - A x in double-float arithmetic on float32 data, row by row in stored
    order: each entry's hi x exactly as a float32 pair (product and its FMA
    remainder), lo x added to the remainder, the running sum kept as an unnormalized
    pair (two-sum of the high parts, the low parts summed), rounded once at the end.
    The float32 steps are numpy float32 operations; the exact remainder of a float32
    product is formed in float64 (where the product is exact) and is a float32."""
    A = A.tocsr()
    n = A.shape[0]
    lens = np.diff(A.indptr)
    w = int(lens.max()) if n else 0
    x = x.astype(f32)
    sh = b.astype(f32).copy()
    sl = np.zeros(n, dtype=f32)
    hi_all, lo_all = split_df(A.data)
    for k in range(w):
        rows = np.nonzero(lens > k)[0]
        pos = A.indptr[rows] + k
        hi, lo = -hi_all[pos], -lo_all[pos]
        xv = x[A.indices[pos]]
        p = hi * xv
        e = (hi.astype(f64) * xv.astype(f64) - p.astype(f64)).astype(f32)
        t = (lo.astype(f64) * xv.astype(f64) + e.astype(f64)).astype(f32)
        s = sh[rows] + p
        bp = s - sh[rows]
        err = (sh[rows] - (s - bp)) + (p - bp)
        sh[rows] = s
        sl[rows] = sl[rows] + (err + t)
    return sh + sl


class EmulatedVcycle:
    def __init__(self, hh, policy, vec=f32):
        self.vec = vec
        self.A = [a.to_scipy().tocsr() for a in hh.A]
        self.P = [p.to_scipy().tocsr() for p in hh.P]
        self.G = [g.to_scipy().tocsr() for g in hh.G]
        self.L = len(self.A)
        self.policy = policy
        self.m, self.maux, self.AG, self.use_ag = [], [], [], []
        for l in range(self.L - 1):
            A, G = self.A[l], self.G[l]
            self.m.append(np.asarray(abs(A).sum(1)).ravel())
            aux = (G.T @ A @ G).tocsr()
            self.maux.append(np.asarray(abs(aux).sum(1)).ravel())
            # A G without the cancellation residue of the floating-point assembly
            AG = (A @ G).tocoo()
            bound = np.asarray((abs(A) @ abs(G)).tocsr()[AG.row, AG.col]).ravel()
            keep = np.abs(AG.data) > 64 * EPS64 * bound
            AG = sp.csr_matrix((AG.data[keep], (AG.row[keep], AG.col[keep])), shape=AG.shape)
            self.AG.append(AG)
            # the CUDA upload's rule: r - (A G) y where it reads fewer bytes than the
            # residual it replaces -- an FP64 residual (A G much sparser than A) in the
            # FP64 V-cycle, a double-float one (up to 1.35 times A's entries) in FP32
            self.use_ag.append(AG.nnz < (1.35 if vec == f32 else 0.6) * A.nnz)
        self.GT = [g.T.tocsr() for g in self.G]
        self.PT = [p.T.tocsr() for p in self.P]
        self._f32 = {}
        for M in self.A + self.P + self.G + self.AG + self.GT + self.PT:
            self._f32[id(M)] = M.astype(f32)
        self.coarse = sla.cho_factor(self.A[-1].toarray(), lower=True)

    def _mv(self, M, x, step, l):
        if self.policy(step, l) == 64:
            return (M @ x.astype(f64)).astype(self.vec)
        return (self._f32[id(M)] @ x.astype(f32)).astype(self.vec)

    def _resid(self, l, step, x, b):
        A = self.A[l]
        if self.policy(step, l) == 48:
            return resid_df(A, x, b).astype(self.vec)
        if self.policy(step, l) == 64:
            return (b.astype(f64) - A @ x.astype(f64)).astype(self.vec)
        return (b.astype(f32) - self._f32[id(A)] @ x.astype(f32)).astype(self.vec)

    def vcycle(self, l, b):
        if l == self.L - 1:
            return sla.cho_solve(self.coarse, b.astype(f64)).astype(self.vec)
        m, ma = self.m[l].astype(self.vec), self.maux[l].astype(self.vec)
        G, GT, P, PT = self.G[l], self.GT[l], self.P[l], self.PT[l]
        x = b / m
        if self.use_ag[l]:
            r = self._resid(l, "pre", x, b)
            y = self._mv(GT, r, "gt", l) / ma
            x = x + self._mv(G, y, "g", l)
            r = r - self._mv(self.AG[l], y, "ag", l)
            e = self.vcycle(l + 1, self._mv(PT, r, "pt", l))
            x = x + self._mv(P, e, "p", l)
            r = self._resid(l, "post", x, b)
            y = self._mv(GT, r, "gt", l) / ma
            x = x + self._mv(G, y, "g", l)
            return x + (r - self._mv(self.AG[l], y, "ag", l)) / m
        r = self._resid(l, "pre", x, b)
        x = x + self._mv(G, self._mv(GT, r, "gt", l) / ma, "g", l)
        r = self._resid(l, "pre2", x, b)
        e = self.vcycle(l + 1, self._mv(PT, r, "pt", l))
        x = x + self._mv(P, e, "p", l)
        r = self._resid(l, "post", x, b)
        x = x + self._mv(G, self._mv(GT, r, "gt", l) / ma, "g", l)
        return x + self._resid(l, "post2", x, b) / m

    def apply(self, r):
        return self.vcycle(0, np.asarray(r, dtype=f64).astype(self.vec)).astype(f64)


def energy_error(A, z, ref):
    """||z - ref||_A / ||ref||_A."""
    d = z - ref
    return float(np.sqrt((d @ (A @ d)) / (ref @ (A @ ref))))
