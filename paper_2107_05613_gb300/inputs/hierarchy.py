"""ctypes binding of the host hierarchy generator (amge_hierarchy.cpp).

The generator builds, on the host in FP64, the AMGe de Rham hierarchy of Sections
2-3 of the paper on an n^3 Kuhn-split unit cube: fine Whitney-form operator A_0,
prolongators P_l from PV traces (eq. 3.5) and local extensions (eqs. 3.6, 3.8),
integer coarse exterior derivatives, and Galerkin operators A_{l+1} = P_l^T A_l P_l.
The result is plain CSR arrays that both the CUDA path and the oracle read.

Levels are numbered from 0 (finest); the paper numbers them from 1.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamge_hierarchy.so")

FORMS = {"hcurl": 1, "hdiv": 2}
KIND_A, KIND_P, KIND_D, KIND_PI, KIND_PIHAT = 0, 1, 2, 3, 4

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from .. import build as _build

        _build.build_hierarchy_lib()
    lib = ctypes.CDLL(LIB_PATH)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.amgh_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.amgh_build.restype = ctypes.c_int
    lib.amgh_error.restype = ctypes.c_char_p
    lib.amgh_num_levels.argtypes = [ctypes.c_void_p]
    lib.amgh_level_counts.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p]
    lib.amgh_matrix_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p]
    lib.amgh_matrix_copy.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.amgh_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    lib.amgh_target_info.argtypes = [ctypes.c_void_p, i64p, ctypes.POINTER(ctypes.c_double)]
    lib.amgh_free.argtypes = [ctypes.c_void_p]
    lib.amgh_free.restype = None
    lib.amgh_fine_assembly_info.argtypes = [ctypes.c_void_p, i64p, ctypes.POINTER(ctypes.c_int)]
    lib.amgh_fine_assembly_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5
    _lib = lib
    return lib


@dataclass
class CSR:
    """Compressed sparse rows: int32 row_ptr / col, float64 values."""

    shape: tuple
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=self.shape)


@dataclass
class Hierarchy:
    """An AMGe hierarchy: per level l, A[l]; per transfer l -> l+1, P[l] and G[l].

    form      'hcurl' (edge dofs, aux space = vertices via the gradient D_0) or
              'hdiv'  (face dofs, aux space = edges via the curl D_1)
    A[l]      problem matrix of level l (paper: A_{l+1})
    P[l]      prolongator of the problem space from level l+1 to level l
    G[l]      aux transition at level l: D_0 (H(curl)) or D_1 (H(div)), integer values
    counts[l] entity counts (vertices, edges, faces, cells)
    P_all[l][k], D_all[l][k]: prolongators / incidences of every space built
    Pi[l][k]  (all_spaces) co-chain projector of space k from level l to l+1
    pihat[l][k] (all_spaces) interpolation of vector H1 (column 3 v + c) into space
              k = 1, 2 at level l (index 0 unused)
    """

    form: str
    n: int
    A: list
    P: list
    G: list
    counts: list
    P_all: list
    D_all: list
    diagnostics: dict
    Pi: list = None
    pihat: list = None

    @property
    def num_levels(self) -> int:
        return len(self.A)


def _copy(lib, h, kind, level, k):
    info = (ctypes.c_int64 * 3)()
    if lib.amgh_matrix_info(h, kind, level, k, info) != 0:
        return None
    nr, nc, nnz = int(info[0]), int(info[1]), int(info[2])
    rp = np.empty(nr + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    rc = lib.amgh_matrix_copy(h, kind, level, k, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    assert rc == 0
    return CSR((nr, nc), rp, ci, v)


def build_hierarchy(form: str, n: int, num_levels: int = 0, beta=None, alpha=None,
                    all_spaces: bool = False, nthreads: int = 0, assembly: bool = False,
                    targets: bool = False) -> Hierarchy:
    """Build the hierarchy on an n^3 Kuhn-split cube (6 n^3 tetrahedra).

    beta, alpha: per-tet coefficients of (Du, Dv) and (u, v) (None = 1).
    num_levels: 0 = coarsen 2x2x2 while the cell grid side m > 8.
    assembly: also return the fine assembly of A_0 as a gather (diagnostics
    "assembly": dict of K, M [6, s, s], coff, ccell, cidx; see amge_hierarchy.h).
    targets: enrich the last coarsening with the degree-one polynomial approximation
    targets (Sections 3.3.1-3.3.3; AMGH_TARGETS in amge_hierarchy.h), or with 2
    (AMGH_TARGETS2) the degree-two ones and the cross-space bubbles of eqs. 3.7 / 3.9:
    P[-1] gains columns after the coarse entities' ones and A[-1] is
    P[-1]^T A[-2] P[-1]; diagnostics "target_functions", "target_constraint".
    """
    lib = _load()
    kf = FORMS[form]
    nt = 6 * n ** 3
    b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    for arr in (b, a):
        if arr is not None and arr.shape != (nt,):
            raise ValueError(f"coefficient array must have {nt} entries")
    h = ctypes.c_void_p()
    deg = int(targets)
    if deg not in (0, 1, 2):
        raise ValueError("targets: False / True (degree one) or 2")
    flags = (1 if all_spaces else 0) | {0: 0, 1: 2, 2: 4}[deg]   # AMGH_ALL_SPACES, AMGH_TARGETS(2)
    rc = lib.amgh_build(kf, n, num_levels, None if b is None else b.ctypes.data,
                        None if a is None else a.ctypes.data, flags, nthreads, ctypes.byref(h))
    if rc != 0:
        raise RuntimeError("hierarchy generator: " + lib.amgh_error().decode())
    try:
        L = lib.amgh_num_levels(h)
        A, P, G, counts, P_all, D_all = [], [], [], [], [], []
        for l in range(L):
            c = (ctypes.c_int64 * 4)()
            lib.amgh_level_counts(h, l, c)
            counts.append(tuple(int(x) for x in c))
            A.append(_copy(lib, h, KIND_A, l, 0))
            D_all.append([_copy(lib, h, KIND_D, l, k) for k in range(3)])
            if l + 1 < L:
                P_all.append([_copy(lib, h, KIND_P, l, k) for k in range(4)])
                P.append(P_all[-1][kf])
                G.append(D_all[-1][kf - 1])
        Pi = pihat = None
        if all_spaces:
            Pi = [[_copy(lib, h, KIND_PI, l, k) for k in range(4)] for l in range(L - 1)]
            pihat = [[None] + [_copy(lib, h, KIND_PIHAT, l, k) for k in (1, 2)] for l in range(L)]
        d = (ctypes.c_double * 4)()
        lib.amgh_diagnostics(h, d)
        diag = {"lambda_dev": d[0], "local_residual": d[1], "incidence_dev": d[2], "seconds": d[3]}
        nf, tc = ctypes.c_int64(), ctypes.c_double()
        lib.amgh_target_info(h, ctypes.byref(nf), ctypes.byref(tc))
        diag["target_functions"], diag["target_constraint"] = nf.value, tc.value
        if assembly:
            nct, sz = ctypes.c_int64(), ctypes.c_int()
            assert lib.amgh_fine_assembly_info(h, ctypes.byref(nct), ctypes.byref(sz)) == 0
            s_ = sz.value
            K = np.empty((6, s_, s_)); M = np.empty((6, s_, s_))
            coff = np.empty(A[0].nnz + 1, np.int32)
            ccell = np.empty(nct.value, np.int32)
            cidx = np.empty(nct.value, np.uint8)
            rc = lib.amgh_fine_assembly_copy(h, K.ctypes.data, M.ctypes.data, coff.ctypes.data, ccell.ctypes.data,
                                             cidx.ctypes.data)
            if rc != 0:
                raise RuntimeError("fine assembly map: " + lib.amgh_error().decode())
            diag["assembly"] = dict(K=K, M=M, coff=coff, ccell=ccell, cidx=cidx, s=s_)
    finally:
        lib.amgh_free(h)
    return Hierarchy(form, n, A, P, G, counts, P_all, D_all, diag, Pi, pihat)


BLOB_MAGIC = b"AMGEBLOB"
BLOB_FORMS = {"hcurl": 2, "hdiv": 3}   # amge_form values (D_2 = curl, D_3 = div)


def _pad8(b: bytes) -> bytes:
    return b + b"\0" * (-len(b) % 8)


def hierarchy_to_blob(h: Hierarchy, nu_pre: int = 1, nu_post: int = 1) -> bytes:
    """Serialize the solve-phase data of a hierarchy (A_l, P_l, G_l) in the blob
    layout of the library's amge_upload_blob: a 32-byte header (magic, version 1,
    form, levels, nu_pre, nu_post, 0), then A_0..A_{L-1}, P_0..P_{L-2}, G_0..G_{L-2},
    each as (int32 rows, int32 cols, int64 nnz, int32 row_ptr, int32 col, float64
    val), little-endian, every section padded to a multiple of 8 bytes."""
    L = h.num_levels
    out = [BLOB_MAGIC, np.array([1], "<u4").tobytes(),
           np.array([BLOB_FORMS[h.form], L, nu_pre, nu_post, 0], "<i4").tobytes()]
    for m in list(h.A) + list(h.P) + list(h.G):
        out.append(np.array(m.shape, "<i4").tobytes() + np.array([m.nnz], "<i8").tobytes())
        out.append(_pad8(np.ascontiguousarray(m.indptr, "<i4").tobytes()))
        out.append(_pad8(np.ascontiguousarray(m.indices, "<i4").tobytes()))
        out.append(np.ascontiguousarray(m.data, "<f8").tobytes())
    return b"".join(out)
