"""Python binding of libamge (the C ABI in include/amge.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device vectors are torch CUDA float64 tensors passed by data pointer;
streams are torch CUDA streams.  If libamge.so has not been built this module
raises on import -- there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

from .build import AMGE_SO

if not os.path.exists(AMGE_SO):
    raise ImportError(
        f"{AMGE_SO} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(there is no CPU fallback for the solve path)")

_lib = ctypes.CDLL(AMGE_SO)

AMGE_OK, AMGE_EINVAL, AMGE_ENOMEM, AMGE_ECUDA, AMGE_ENOTCONV, AMGE_ENONFINITE = 0, 1, 2, 3, 4, 5
AMGE_EAGAIN, AMGE_ETIMEOUT, AMGE_ECANCELED = 6, 7, 8
AMGE_HCURL, AMGE_HDIV = 2, 3
AMGE_SETUP_TARGETS, AMGE_SETUP_TARGETS2 = 1, 2
AMGE_FP64, AMGE_FP32_VCYCLE = 0, 1
AMGE_OP_A, AMGE_OP_P, AMGE_OP_PT, AMGE_OP_G, AMGE_OP_GT, AMGE_OP_SMOOTH_PRE, AMGE_OP_COARSE, AMGE_OP_AG, AMGE_OP_A_WIDE = range(9)
PROF_CLASSES = ["A_fine", "A_coarse", "GT", "G", "PT", "P", "coarse", "pcg_spmv", "pcg_vec", "vcycle_vec", "AG",
                "A_wide", "gs"]
AMGE_SMOOTHER_L1_JACOBI, AMGE_SMOOTHER_SYM_GS = 0, 1
AMGE_WIDE_FP64, AMGE_WIDE_DF = 0, 1
AMGE_COARSE_DENSE, AMGE_COARSE_AUX = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ENONFINITE",
                6: "EAGAIN", 7: "ETIMEOUT", 8: "ECANCELED"}


class amge_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class amge_hierarchy_desc(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("A", ctypes.POINTER(amge_csr)), ("P", ctypes.POINTER(amge_csr)),
                ("G", ctypes.POINTER(amge_csr)), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32)]


class amge_problem(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("n", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("beta", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("nu_pre", ctypes.c_int32),
                ("nu_post", ctypes.c_int32), ("flags", ctypes.c_int32)]


class amge_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32), ("precision", ctypes.c_int32)]


class amge_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("true_relres", ctypes.c_double),
                ("time_ms", ctypes.c_double)]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "amge_setup_upload": [ctypes.POINTER(amge_problem), _vp, ctypes.POINTER(_vp)],
    "amge_upload_blob": [_vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
    "amge_upload_levels": [ctypes.POINTER(amge_hierarchy_desc), _vp, ctypes.POINTER(_vp)],
    "amge_hier_info": [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_size_t)],
    "amge_vcycle": [_vp, _vp, _vp, _i32, _i32, _vp],
    "amge_pcg_solve": [_vp, _vp, _vp, _i32, ctypes.POINTER(amge_solve_opts), ctypes.POINTER(amge_info), _vp],
    "amge_pcg_solve_host": [_vp, _vp, _vp, _i32, ctypes.POINTER(amge_solve_opts), ctypes.POINTER(amge_info),
                            _vp],
    "amge_apply": [_vp, _i32, _i32, _vp, _vp, _i32, _vp],
    "amge_dot": [_vp, _vp, _vp, _i64, _vp, _vp],
    "amge_profile_enable": [_vp, _i32],
    "amge_set_graphs": [_vp, _i32],
    "amge_autotune_report": [_vp, ctypes.POINTER(_i32)],
    "amge_set_kernel": [_vp, _i32, _i32, _i32, _i32],
    "amge_autotune_times": [_vp, ctypes.POINTER(ctypes.c_float)],
    "amge_server_create": [ctypes.c_size_t, _i32, ctypes.POINTER(_vp)],
    "amge_submit": [_vp, _vp, _vp, _vp, _i32, ctypes.POINTER(amge_solve_opts), ctypes.POINTER(ctypes.c_uint64)],
    "amge_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(amge_info)],
    "amge_wait": [_vp, ctypes.c_uint64, _i32, ctypes.POINTER(amge_info)],
    "amge_cancel": [_vp, ctypes.c_uint64],
    "amge_server_stats": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_size_t),
                          ctypes.POINTER(_i32)],
    "amge_profile_read": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)],
    "amge_coarse_solve_noalloc": [_vp, _vp, _vp, _vp],
    "amge_fp64_fma_rate": [ctypes.POINTER(ctypes.c_double), _vp],
    "amge_fp64_mma_rate": [ctypes.POINTER(ctypes.c_double), _vp],
    "amge_autotune_report_mm": [_vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)],
    "amge_set_kernel_mm": [_vp, _i32, _i32, _i32, _i32, _i32],
    "amge_set_smoother": [_vp, _i32, _i32, _i32],
    "amge_update_coefficients": [_vp, _vp, _vp, _vp],
    "amge_wait_status": [_vp, _vp, ctypes.POINTER(_i32)],
    "amge_set_wide_arith": [_vp, _i32],
    "amge_pcg_kernel": [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)],
    "amge_set_coarse_solver": [_vp, _i32, _i32, ctypes.POINTER(amge_csr), ctypes.POINTER(amge_csr),
                               ctypes.POINTER(amge_csr), _vp],
    "amge_df_form": [_vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_i32)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.amge_set_dependent_launch.argtypes = [_i32]
_lib.amge_set_dependent_launch.restype = None
_lib.amge_hier_free.argtypes = [_vp]
_lib.amge_hier_free.restype = None
_lib.amge_server_destroy.argtypes = [_vp]
_lib.amge_server_destroy.restype = None
_lib.amge_last_error.argtypes = []
_lib.amge_last_error.restype = ctypes.c_char_p


class AmgeError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {amge_last_error()}")


def amge_last_error() -> str:
    return _lib.amge_last_error().decode()


def _check(st, where, allow=(AMGE_OK,)):
    if st not in allow:
        raise AmgeError(st, where)
    return st


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, n=None):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("device vectors must be contiguous CUDA float64 tensors")
    if n is not None and t.numel() < n:
        raise ValueError(f"device vector has {t.numel()} entries, needs {n}")
    return ctypes.c_void_p(t.data_ptr())


class Hier:
    """Owning handle of an uploaded hierarchy (freed with amge_hier_free)."""

    def __init__(self, handle, n, levels):
        self.handle = handle
        self.n = n
        self.levels = levels

    def free(self):
        if self.handle:
            _lib.amge_hier_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def _csr_struct(m, keep):
    rp = np.ascontiguousarray(m.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(m.indices, dtype=np.int32)
    v = np.ascontiguousarray(m.data, dtype=np.float64)
    keep += [rp, ci, v]
    return amge_csr(m.shape[0], m.shape[1], int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)


def _hier_from(h):
    n, lv, nb = amge_hier_info(h)
    return Hier(h, n, lv)


def amge_setup_upload(form: str, n: int, num_levels: int = 0, beta=None, alpha=None, nu_pre: int = 1,
                      nu_post: int = 1, stream=None, targets: bool = False, flags: int = None) -> Hier:
    """Build the hierarchy of the problem (eq. 2.2 on n^3 Kuhn-split cubes) on the host
    and upload it.  form: 'hcurl' or 'hdiv'; beta / alpha: per-tet coefficients of the
    derivative / mass term (6 n^3 values, None = 1); targets: True / 1 for
    AMGE_SETUP_TARGETS, 2 for AMGE_SETUP_TARGETS2 (flags, when given, is passed as it
    is)."""
    keep = []

    def coef(c):
        if c is None:
            return None
        a = np.ascontiguousarray(c, dtype=np.float64)
        if a.size != 6 * n ** 3:
            raise ValueError(f"coefficient array must have {6 * n ** 3} entries")
        keep.append(a)
        return a.ctypes.data

    if flags is None:
        flags = {0: 0, 1: AMGE_SETUP_TARGETS, 2: AMGE_SETUP_TARGETS2}[int(targets)]
    prob = amge_problem({"hcurl": AMGE_HCURL, "hdiv": AMGE_HDIV}[form], n, num_levels, coef(beta), coef(alpha),
                        nu_pre, nu_post, flags)
    h = ctypes.c_void_p()
    _check(_lib.amge_setup_upload(ctypes.byref(prob), _stream(stream), ctypes.byref(h)), "amge_setup_upload")
    return _hier_from(h)


def amge_upload_blob(blob: bytes, stream=None) -> Hier:
    """Upload a hierarchy serialized in the blob format of include/amge.h."""
    buf = np.frombuffer(blob, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(_lib.amge_upload_blob(buf.ctypes.data, buf.size, _stream(stream), ctypes.byref(h)), "amge_upload_blob")
    return _hier_from(h)


def amge_upload_levels(hierarchy, stream=None, nu_pre: int = 1, nu_post: int = 1) -> Hier:
    """Upload an inputs.Hierarchy (or any object with form, A, P, G lists of CSR)."""
    keep = []
    L = len(hierarchy.A)
    A = (amge_csr * L)(*[_csr_struct(a, keep) for a in hierarchy.A])
    P = (amge_csr * max(L - 1, 1))(*[_csr_struct(p, keep) for p in hierarchy.P])
    G = (amge_csr * max(L - 1, 1))(*[_csr_struct(g, keep) for g in hierarchy.G])
    form = {"hcurl": AMGE_HCURL, "hdiv": AMGE_HDIV}[hierarchy.form]
    desc = amge_hierarchy_desc(form, L, A, P, G, nu_pre, nu_post)
    h = ctypes.c_void_p()
    _check(_lib.amge_upload_levels(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "amge_upload_levels")
    return _hier_from(h)


def amge_hier_info(h):
    handle = h.handle if isinstance(h, Hier) else h
    n, lv, nb = _i32(), _i32(), ctypes.c_size_t()
    _check(_lib.amge_hier_info(handle, ctypes.byref(n), ctypes.byref(lv), ctypes.byref(nb)), "amge_hier_info")
    return n.value, lv.value, nb.value


def amge_vcycle(h: Hier, r, z, nrhs: int = 1, precision: int = AMGE_FP64, stream=None):
    _check(_lib.amge_vcycle(h.handle, _dptr(r, h.n * nrhs), _dptr(z, h.n * nrhs), nrhs, precision,
                            _stream(stream)), "amge_vcycle")


def amge_pcg_solve(h: Hier, b, x, rtol=1e-8, maxit=1000, precision=AMGE_FP64, nrhs=1, stream=None):
    """Returns (status, [info dicts])."""
    opts = amge_solve_opts(rtol, maxit, precision)
    infos = (amge_info * nrhs)()
    st = _lib.amge_pcg_solve(h.handle, _dptr(b, h.n * nrhs), _dptr(x, h.n * nrhs), nrhs, ctypes.byref(opts),
                             infos, _stream(stream))
    _check(st, "amge_pcg_solve", allow=(AMGE_OK, AMGE_ENOTCONV, AMGE_ENONFINITE))
    return st, [dict(iters=i.iters, status=i.status, true_relres=i.true_relres, time_ms=i.time_ms) for i in infos]


def amge_pcg_solve_host(h: Hier, b_host, x_host, rtol=1e-8, maxit=1000, precision=AMGE_FP64, nrhs=1,
                        stream=None):
    """Host-buffer solve: b_host / x_host are CPU float64 tensors or numpy arrays."""
    def hptr(a):
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size >= h.n * nrhs
            return ctypes.c_void_p(a.ctypes.data)
        assert (not a.is_cuda) and a.is_contiguous() and a.numel() >= h.n * nrhs
        return ctypes.c_void_p(a.data_ptr())

    opts = amge_solve_opts(rtol, maxit, precision)
    infos = (amge_info * nrhs)()
    st = _lib.amge_pcg_solve_host(h.handle, hptr(b_host), hptr(x_host), nrhs, ctypes.byref(opts), infos,
                                  _stream(stream))
    _check(st, "amge_pcg_solve_host", allow=(AMGE_OK, AMGE_ENOTCONV, AMGE_ENONFINITE))
    return st, [dict(iters=i.iters, status=i.status, true_relres=i.true_relres, time_ms=i.time_ms) for i in infos]


def amge_apply(h: Hier, op: int, level: int, x, y, precision=AMGE_FP64, stream=None):
    _check(_lib.amge_apply(h.handle, op, level, _dptr(x), _dptr(y), precision, _stream(stream)), "amge_apply")


def amge_dot(h: Hier, x, y, n: int, out, stream=None):
    _check(_lib.amge_dot(h.handle, _dptr(x, n), _dptr(y, n), n, _dptr(out, 1), _stream(stream)), "amge_dot")


def amge_coarse_solve_noalloc(h: Hier, b, z, stream=None):
    """Coarsest-level solve whose intermediate vector lives in a fixed device array
    (no allocation by the library during the call); see include/amge.h."""
    _check(_lib.amge_coarse_solve_noalloc(h.handle, _dptr(b), _dptr(z), _stream(stream)),
           "amge_coarse_solve_noalloc")


def amge_autotune_report(h: Hier):
    """{(level, 'fp64'|'fp32', op): code} -- 0 = sliced ELL, 100 w = sliced ELL with w warps
    per slice, k <= 32 = vector CSR with k lanes/row, -1 = operator not stored."""
    L = h.levels
    buf = (_i32 * max((L - 1) * 12, 1))()
    _check(_lib.amge_autotune_report(h.handle, buf), "amge_autotune_report")
    ops = ["A", "P", "PT", "G", "GT", "AG"]
    return {(l, p, ops[o]): int(buf[(l * 2 + pi) * 6 + o]) for l in range(L - 1)
            for pi, p in enumerate(("fp64", "fp32")) for o in range(6)}


OPS = ["A", "P", "PT", "G", "GT", "AG"]
TUNE_CODES = [0, 200, 400, 800, 2, 4, 8, 16, 32, 1000, 1200, 3000, 1600, 1700, 1800, 1900, 2000]


def amge_autotune_times(h: Hier):
    """{(level, 'fp64'|'fp32', op): {code: us per launch}} as measured at upload."""
    L = h.levels
    buf = (ctypes.c_float * max((L - 1) * 204, 1))()
    _check(_lib.amge_autotune_times(h.handle, buf), "amge_autotune_times")
    out = {}
    for l in range(L - 1):
        for pi, p in enumerate(("fp64", "fp32")):
            for o in range(6):
                t = {c: round(float(buf[((l * 2 + pi) * 6 + o) * 17 + k]), 2) for k, c in enumerate(TUNE_CODES)}
                if any(v >= 0 for v in t.values()):
                    out[(l, p, OPS[o])] = {c: v for c, v in t.items() if v >= 0}
    return out


def amge_set_kernel(h: Hier, level: int, precision, op, lanes: int):
    """Pin the kernel of one operator: lanes 0 = sliced ELL, 200/400/800 = sliced ELL
    with 2/4/8 warps per slice, 2..32 = vector CSR with that many lanes per row.
    precision: 0/1 or 'fp64'/'fp32'; op: index or name from OPS."""
    p = {"fp64": 0, "fp32": 1}.get(precision, precision)
    o = OPS.index(op) if isinstance(op, str) else op
    _check(_lib.amge_set_kernel(h.handle, level, int(p), int(o), lanes), "amge_set_kernel")


def amge_set_dependent_launch(enable: bool = True):
    """Process-wide programmatic dependent launch of the library's kernels (default on)."""
    _lib.amge_set_dependent_launch(int(enable))


def amge_set_wide_arith(h: Hier, arith: int):
    """Arithmetic of the FP32 V-cycle's residuals of corrected iterates:
    AMGE_WIDE_DF (double-float on the FP32 pipe, default) or AMGE_WIDE_FP64."""
    _check(_lib.amge_set_wide_arith(h.handle, int(arith)), "amge_set_wide_arith")


def amge_pcg_kernel(h: Hier, code=None):
    """The PCG product's kernel (0, 1700 or 1000) and the upload-time timings [us for 0,
    1700, 1000]; with `code`, set it first."""
    c = _i32(0 if code is None else int(code))
    us = (ctypes.c_float * 3)()
    _check(_lib.amge_pcg_kernel(h.handle, 0 if code is None else 1, ctypes.byref(c), us), "amge_pcg_kernel")
    return c.value, [round(float(u), 2) for u in us]


def amge_df_form(h: Hier, level: int, form=None, layout: bool = False):
    """The double-float product's form on a smoothing level (0 32-bit columns, 1 16-bit,
    2 16-bit with L2 prefetch) and the upload-time timings; with `form`, set it first.
    layout=True also returns the 16-bit column layout (0 none, 1 per-slice base, 2 per-row)."""
    f = _i32(0 if form is None else int(form))
    us = (ctypes.c_float * 3)()
    lay = _i32(0)
    _check(_lib.amge_df_form(h.handle, level, 0 if form is None else 1, ctypes.byref(f), us, ctypes.byref(lay)),
           "amge_df_form")
    out = (f.value, [round(float(u), 2) for u in us])
    return out + (lay.value,) if layout else out


def amge_set_coarse_solver(h: Hier, solver: int, iters: int = 5, pihat=None, D=None, pihat_inner=None,
                           stream=None):
    """Coarsest solver: AMGE_COARSE_DENSE or AMGE_COARSE_AUX (iters PCG iterations with
    the auxiliary-space preconditioner of eq. 4.2; pihat, D, pihat_inner: CSR matrices
    of the coarsest level, see amge_coarse_aux_inputs)."""
    keep = []
    ptr = lambda m: None if m is None else ctypes.pointer(_csr_struct(m, keep))
    _check(_lib.amge_set_coarse_solver(h.handle, int(solver), int(iters), ptr(pihat), ptr(D), ptr(pihat_inner),
                                       _stream(stream)), "amge_set_coarse_solver")


def amge_coarse_aux_inputs(hierarchy):
    """(pihat, D, pihat_inner) of the coarsest level of a generated hierarchy built with
    all spaces: the vector-H1 interpolation into the problem space, the exterior
    derivative into it, and (H(div)) the interpolation into the edge space."""
    L = hierarchy.num_levels
    if hierarchy.pihat is None:
        raise ValueError("the hierarchy was built without all spaces")
    if hierarchy.form == "hcurl":
        return hierarchy.pihat[L - 1][1], hierarchy.D_all[L - 1][0], None
    return hierarchy.pihat[L - 1][2], hierarchy.D_all[L - 1][1], hierarchy.pihat[L - 1][1]


def amge_wait_status(h: Hier, stream=None) -> bool:
    """True if a kernel of h with bounded waits (the bulk-staged product) ran out of
    time since the previous check (the results since then are not valid); clears it."""
    v = _i32()
    _check(_lib.amge_wait_status(h.handle, _stream(stream), ctypes.byref(v)), "amge_wait_status")
    return bool(v.value)


def amge_set_graphs(h: Hier, enable: bool = True):
    """Graph-driven (True) or host-launched (False) single-RHS PCG iterations."""
    _check(_lib.amge_set_graphs(h.handle, int(enable)), "amge_set_graphs")


def amge_profile_enable(h: Hier, enable: bool = True):
    _check(_lib.amge_profile_enable(h.handle, int(enable)), "amge_profile_enable")


def amge_profile_read(h: Hier):
    """{class name: (launches, total ms)} since the previous read."""
    cnt = (_i64 * len(PROF_CLASSES))()
    ms = (ctypes.c_double * len(PROF_CLASSES))()
    _check(_lib.amge_profile_read(h.handle, cnt, ms), "amge_profile_read")
    return {name: (int(cnt[i]), float(ms[i])) for i, name in enumerate(PROF_CLASSES)}


class Server:
    """Owning handle of a request server (amge_server_create / amge_server_destroy).

    Keeps every submitted request's host buffers alive until its result is collected.
    """

    def __init__(self, handle):
        self.handle = handle
        self._live = {}

    def destroy(self):
        if self.handle:
            _lib.amge_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:  # noqa: BLE001
            pass


def amge_server_create(hbm_budget_bytes: int = 0, max_slots: int = 16) -> Server:
    h = ctypes.c_void_p()
    _check(_lib.amge_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h)), "amge_server_create")
    return Server(h)


def amge_submit(sv: Server, h: Hier, b_host, x_host, nrhs: int = 1, rtol=1e-8, maxit=1000, precision=AMGE_FP64):
    """b_host / x_host: C-contiguous float64 numpy arrays of n*nrhs entries.  Returns a ticket."""
    assert b_host.dtype == np.float64 and b_host.flags.c_contiguous and b_host.size == h.n * nrhs
    assert x_host.dtype == np.float64 and x_host.flags.c_contiguous and x_host.size == h.n * nrhs
    opts = amge_solve_opts(rtol, maxit, precision)
    t = ctypes.c_uint64()
    _check(_lib.amge_submit(sv.handle, h.handle, ctypes.c_void_p(b_host.ctypes.data),
                            ctypes.c_void_p(x_host.ctypes.data), nrhs, ctypes.byref(opts), ctypes.byref(t)),
           "amge_submit")
    sv._live[t.value] = (b_host, x_host, nrhs, h)
    return t.value


def _collect(sv, ticket, st, infos, nrhs):
    sv._live.pop(ticket, None)
    return st, [dict(iters=i.iters, status=i.status, true_relres=i.true_relres, time_ms=i.time_ms)
                for i in infos[:nrhs]]


def amge_poll(sv: Server, ticket: int):
    """(AMGE_EAGAIN, None) while pending, else (status, [info per column])."""
    nrhs = sv._live[ticket][2] if ticket in sv._live else kMaxRhs
    infos = (amge_info * max(nrhs, 1))()
    st = _lib.amge_poll(sv.handle, ticket, infos)
    if st == AMGE_EAGAIN:
        return st, None
    _check(st, "amge_poll", allow=(AMGE_OK, AMGE_ENOTCONV, AMGE_ENONFINITE, AMGE_ECANCELED, AMGE_ENOMEM, AMGE_ECUDA))
    return _collect(sv, ticket, st, infos, nrhs)


def amge_wait(sv: Server, ticket: int, timeout_ms: int = -1):
    nrhs = sv._live[ticket][2] if ticket in sv._live else kMaxRhs
    infos = (amge_info * max(nrhs, 1))()
    st = _lib.amge_wait(sv.handle, ticket, timeout_ms, infos)
    if st == AMGE_ETIMEOUT:
        return st, None
    _check(st, "amge_wait", allow=(AMGE_OK, AMGE_ENOTCONV, AMGE_ENONFINITE, AMGE_ECANCELED, AMGE_ENOMEM, AMGE_ECUDA))
    return _collect(sv, ticket, st, infos, nrhs)


def amge_cancel(sv: Server, ticket: int):
    _check(_lib.amge_cancel(sv.handle, ticket), "amge_cancel")


def amge_server_stats(sv: Server):
    q, r, nb, ns = _i64(), _i64(), ctypes.c_size_t(), _i32()
    _check(_lib.amge_server_stats(sv.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(nb), ctypes.byref(ns)),
           "amge_server_stats")
    return dict(queued=q.value, running_columns=r.value, bytes_in_use=nb.value, slots=ns.value)


def amge_server_destroy(sv: Server):
    sv.destroy()


kMaxRhs = 32


def lib_handle():
    """The loaded ctypes library (tests inspect its exports)."""
    return _lib


def amge_fp64_fma_rate(stream=None) -> float:
    """FP64 FMA issue rate of the current device, TFMA/s."""
    v = ctypes.c_double()
    _check(_lib.amge_fp64_fma_rate(ctypes.byref(v), _stream(stream)), "amge_fp64_fma_rate")
    return v.value


_OPS = ["A", "P", "PT", "G", "GT", "AG"]


def amge_autotune_report_mm(h: Hier, nrhs: int, precision: int = AMGE_FP32_VCYCLE):
    """({(level, op): code}, {(level, op): [us CSR, us sliced ELL x1, us x2]}) of the block
    products for nrhs columns: 0 = CSR, 1 / 2 = sliced ELL with 1 / 2 vectors per lane,
    -1 = not stored / not tuned yet; key (levels-1, "coarse"): the coarsest product, 0 =
    CUDA cores, 1 = FP64 tensor cores, with [us CUDA cores, us tensor cores]."""
    L = h.levels
    codes = (_i32 * ((L - 1) * 6 + 1))()
    us = (ctypes.c_float * ((L - 1) * 18 + 3))()
    _check(_lib.amge_autotune_report_mm(h.handle, nrhs, precision, codes, us), "amge_autotune_report_mm")
    c = {(l, _OPS[o]): int(codes[l * 6 + o]) for l in range(L - 1) for o in range(6)}
    t = {(l, _OPS[o]): [float(us[(l * 6 + o) * 3 + k]) for k in range(3)] for l in range(L - 1) for o in range(6)}
    c[(L - 1, "coarse")] = int(codes[(L - 1) * 6])      # 0 CUDA cores, 1 FP64 tensor cores
    t[(L - 1, "coarse")] = [float(us[(L - 1) * 18 + k]) for k in range(2)]
    return c, t


def amge_set_kernel_mm(h: Hier, level: int, precision: int, op, nrhs: int, code: int):
    """op "coarse" (6): the coarsest product, code 0 CUDA cores / 1 FP64 tensor cores."""
    o = (6 if op == "coarse" else _OPS.index(op)) if isinstance(op, str) else op
    _check(_lib.amge_set_kernel_mm(h.handle, level, precision, o, nrhs, code), "amge_set_kernel_mm")


def amge_set_smoother(h: Hier, smoother: int, sweeps: int = 2, gs_levels: int = 64):
    """AMGE_SMOOTHER_L1_JACOBI, or AMGE_SMOOTHER_SYM_GS (`sweeps` symmetric Gauss-Seidel
    steps per smoothing) on the gs_levels finest smoothing levels."""
    _check(_lib.amge_set_smoother(h.handle, smoother, sweeps, gs_levels), "amge_set_smoother")


def amge_update_coefficients(h: Hier, beta=None, alpha=None, stream=None):
    """New per-tetrahedron coefficients for a hierarchy made by amge_setup_upload (GPU
    re-setup of the Galerkin operators; see include/amge.h)."""
    keep = []

    def ptr(c):
        if c is None:
            return None
        a = np.ascontiguousarray(c, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data

    _check(_lib.amge_update_coefficients(h.handle, ptr(beta), ptr(alpha), _stream(stream)),
           "amge_update_coefficients")


def amge_fp64_mma_rate(stream=None) -> float:
    """FP64 tensor-core (mma.sync m8n8k4) rate of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(_lib.amge_fp64_mma_rate(ctypes.byref(v), _stream(stream)), "amge_fp64_mma_rate")
    return v.value
