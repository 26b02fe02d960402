"""The problem-level setup entry points on the CPU (no GPU is touched).

* amge_setup_upload validates the problem of eq. 2.2 (form, n, levels, smoothing
  steps, positive finite coefficients) and returns AMGE_EINVAL before any work; a
  valid problem reaches the device step first (AMGE_ECUDA without a GPU) before the
  host setup runs.
* The hierarchy blob: the writer of the inputs module and the oracle's independent
  reader agree bit for bit with the generated matrices; the library's reader rejects
  malformed blobs (magic, version, level count, truncation, trailing bytes) with
  AMGE_EINVAL and hands a valid one on to the upload (AMGE_ECUDA without a GPU).
"""
import ctypes
import os

import numpy as np
import pytest

from conftest import hierarchy
from oracle import OracleHierarchy
from paper_2107_05613_gb300.inputs import hierarchy_to_blob

AMGE_EINVAL, AMGE_ECUDA = 1, 3
AMGE_HCURL, AMGE_HDIV = 2, 3


class Problem(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("n", ctypes.c_int32), ("num_levels", ctypes.c_int32),
                ("beta", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("nu_pre", ctypes.c_int32),
                ("nu_post", ctypes.c_int32)]


@pytest.fixture(scope="module")
def lib():
    from paper_2107_05613_gb300 import build

    if not os.path.exists(build.AMGE_SO):
        build.build_amge_lib()
    lib = ctypes.CDLL(build.AMGE_SO)
    lib.amge_setup_upload.restype = ctypes.c_int
    lib.amge_setup_upload.argtypes = [ctypes.POINTER(Problem), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.amge_upload_blob.restype = ctypes.c_int
    lib.amge_upload_blob.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    lib.amge_last_error.restype = ctypes.c_char_p
    return lib


def _gpu_absent():
    try:
        import torch

        return not torch.cuda.is_available()
    except ImportError:
        return True


def test_setup_upload_rejects_bad_problems(lib):
    n = 2
    good = np.ones(6 * n ** 3)
    neg = good.copy()
    neg[5] = -1.0
    nan = good.copy()
    nan[0] = np.nan
    cases = [dict(form=1), dict(form=4), dict(n=0), dict(n=257), dict(num_levels=-1), dict(num_levels=17),
             dict(nu_pre=0), dict(nu_post=9), dict(beta=neg), dict(alpha=nan)]
    for c in cases:
        args = dict(form=AMGE_HCURL, n=n, num_levels=0, beta=None, alpha=None, nu_pre=1, nu_post=1)
        args.update(c)
        b = args["beta"]
        a = args["alpha"]
        p = Problem(args["form"], args["n"], args["num_levels"], None if b is None else b.ctypes.data,
                    None if a is None else a.ctypes.data, args["nu_pre"], args["nu_post"])
        out = ctypes.c_void_p(1)
        assert lib.amge_setup_upload(ctypes.byref(p), None, ctypes.byref(out)) == AMGE_EINVAL, c
        assert out.value is None
    out = ctypes.c_void_p()
    assert lib.amge_setup_upload(None, None, ctypes.byref(out)) == AMGE_EINVAL
    assert lib.amge_setup_upload(ctypes.byref(Problem(AMGE_HDIV, 2, 0, None, None, 1, 1)), None, None) == AMGE_EINVAL


@pytest.mark.skipif(not _gpu_absent(), reason="checks the no-device path")
def test_setup_upload_checks_the_device_before_the_host_setup(lib):
    p = Problem(AMGE_HCURL, 4, 0, None, None, 1, 1)
    out = ctypes.c_void_p()
    assert lib.amge_setup_upload(ctypes.byref(p), None, ctypes.byref(out)) == AMGE_ECUDA
    assert out.value is None


@pytest.mark.parametrize("form,n,L", [("hcurl", 4, 2), ("hdiv", 4, 3), ("hcurl", 2, 1)])
def test_blob_round_trip_through_the_oracle_reader(form, n, L):
    hh = hierarchy(form, n, L, True)
    blob = hierarchy_to_blob(hh, nu_pre=1, nu_post=1)
    assert len(blob) % 8 == 0
    o = OracleHierarchy.from_blob(blob)
    ref = OracleHierarchy.from_hierarchy(hh)
    assert o.L == ref.L == L
    for mine, theirs in zip(o.A + o.P + o.G, ref.A + ref.P + ref.G):
        assert mine.shape == theirs.shape
        assert (mine != theirs).nnz == 0
        assert np.array_equal(mine.indptr, theirs.indptr) and np.array_equal(mine.indices, theirs.indices)
        assert np.array_equal(mine.data, theirs.data)
    with pytest.raises(ValueError):
        OracleHierarchy.from_blob(blob + b"\0" * 8)


def test_library_blob_reader(lib):
    hh = hierarchy("hcurl", 4, 2, True)
    blob = bytearray(hierarchy_to_blob(hh))

    def call(b, size=None):
        buf = (ctypes.c_ubyte * max(len(b), 1)).from_buffer_copy(bytes(b) or b"\0")
        out = ctypes.c_void_p(1)
        st = lib.amge_upload_blob(ctypes.addressof(buf), len(b) if size is None else size, None, ctypes.byref(out))
        if st != 0:
            assert out.value is None
        return st

    bad_magic = bytearray(blob)
    bad_magic[0] ^= 1
    bad_version = bytearray(blob)
    bad_version[8] = 2
    bad_levels = bytearray(blob)
    bad_levels[16:20] = (17).to_bytes(4, "little")
    huge_nnz = bytearray(blob)
    huge_nnz[40:48] = (1 << 40).to_bytes(8, "little")
    for b in (bad_magic, bad_version, bad_levels, huge_nnz, blob[:-8], blob[:31], blob + b"\0" * 8, b""):
        assert call(b) == AMGE_EINVAL
        assert b"blob" in lib.amge_last_error()
    out = ctypes.c_void_p()
    assert lib.amge_upload_blob(None, 0, None, ctypes.byref(out)) == AMGE_EINVAL
    if _gpu_absent():
        assert call(blob) == AMGE_ECUDA          # parsed; the upload needs a device
        # an unaligned copy of the blob is read the same way
        shifted = (ctypes.c_ubyte * (len(blob) + 1))()
        ctypes.memmove(ctypes.addressof(shifted) + 1, bytes(blob), len(blob))
        assert lib.amge_upload_blob(ctypes.addressof(shifted) + 1, len(blob), None, ctypes.byref(out)) == AMGE_ECUDA
