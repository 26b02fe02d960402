"""From coefficients to a solved system through the C ABI alone (ctypes on libamge.so).

The problem of eq. 2.2 -- H(curl) and H(div) on 16^3 Kuhn-split cubes, the derivative
coefficient beta log-uniform in [1e-3, 1e3] per 8^3 block, alpha = 1 -- goes in as
coefficients (amge_setup_upload: host FP64 setup of Sections 2-3, then the upload),
and as a serialized hierarchy (amge_upload_blob); both are solved with
amge_pcg_solve_host on host buffers.  No Python arithmetic touches the solve: the
test only marshals arrays.  The oracle solves the same problem from the generator's
hierarchy (and from the same blob): iterations within 1, solution within 1e-9.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMGE_HCURL, AMGE_HDIV = 2, 3


class Problem(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("n", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("beta", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("nu_pre", ctypes.c_int32),
                ("nu_post", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32), ("precision", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("true_relres", ctypes.c_double),
                ("time_ms", ctypes.c_double)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05613_gb300 import build

    torch.cuda.init()
    lib = ctypes.CDLL(build.AMGE_SO)
    vp = ctypes.c_void_p
    lib.amge_setup_upload.argtypes = [ctypes.POINTER(Problem), vp, ctypes.POINTER(vp)]
    lib.amge_upload_blob.argtypes = [vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    lib.amge_pcg_solve_host.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.POINTER(Opts), ctypes.POINTER(Info), vp]
    lib.amge_hier_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_size_t)]
    lib.amge_hier_free.argtypes = [vp]
    lib.amge_hier_free.restype = None
    lib.amge_last_error.restype = ctypes.c_char_p
    for f in (lib.amge_setup_upload, lib.amge_upload_blob, lib.amge_pcg_solve_host, lib.amge_hier_info):
        f.restype = ctypes.c_int
    return lib


def _solve(lib, h, b, precision=0):
    n = ctypes.c_int32()
    levels = ctypes.c_int32()
    assert lib.amge_hier_info(h, ctypes.byref(n), ctypes.byref(levels), None) == 0
    assert n.value == b.size
    x = np.zeros_like(b)
    info = Info()
    st = lib.amge_pcg_solve_host(h, b.ctypes.data, x.ctypes.data, 1, ctypes.byref(Opts(1e-8, 1000, precision)),
                                 ctypes.byref(info), None)
    assert st == 0, lib.amge_last_error()
    return x, info, levels.value


@pytest.mark.parametrize("form", ["hcurl", "hdiv"])
def test_coefficients_to_solution_through_the_abi(lib, form):
    from oracle import OracleHierarchy, pcg
    from paper_2107_05613_gb300.inputs import build_hierarchy, hierarchy_to_blob, rhs_vector
    from paper_2107_05613_gb300.inputs.rng import workload_coefficients

    n = 16
    beta, alpha = workload_coefficients(n, True, 2107056137)
    beta = np.ascontiguousarray(beta)
    alpha = np.ascontiguousarray(alpha)
    prob = Problem(AMGE_HCURL if form == "hcurl" else AMGE_HDIV, n, 0, beta.ctypes.data, alpha.ctypes.data, 1, 1)
    h = ctypes.c_void_p()
    assert lib.amge_setup_upload(ctypes.byref(prob), None, ctypes.byref(h)) == 0, lib.amge_last_error()

    hh = build_hierarchy(form, n, 0, beta, alpha)
    b = rhs_vector(2107056138, hh.A[0].shape[0])
    o = OracleHierarchy.from_hierarchy(hh)
    xo, it_o, _, ok = pcg(o, b, rtol=1e-8)
    assert ok
    x, info, levels = _solve(lib, h, b)
    lib.amge_hier_free(h)
    assert levels == o.L == 2
    assert abs(info.iters - it_o) <= 1 and info.true_relres <= 1e-8
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)

    blob = hierarchy_to_blob(hh)
    buf = np.frombuffer(blob, dtype=np.uint8)
    h = ctypes.c_void_p()
    assert lib.amge_upload_blob(buf.ctypes.data, buf.size, None, ctypes.byref(h)) == 0, lib.amge_last_error()
    ob = OracleHierarchy.from_blob(blob)
    xb_o, itb_o, _, _ = pcg(ob, b, rtol=1e-8)
    assert itb_o == it_o and np.array_equal(xb_o, xo)      # same data, same oracle result
    x, info, _ = _solve(lib, h, b)
    assert abs(info.iters - it_o) <= 1 and info.true_relres <= 1e-8
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    x32, info32, _ = _solve(lib, h, b, precision=1)
    assert info32.true_relres <= 1e-8 and info32.iters <= it_o + 3
    lib.amge_hier_free(h)
