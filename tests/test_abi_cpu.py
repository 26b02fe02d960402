"""The C ABI library loads and exports every symbol include/amge.h declares.

No GPU is touched: only argument-validation paths that return before any CUDA call.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_05613_gb300 import build

    if not os.path.exists(build.AMGE_SO):
        build.build_amge_lib()
    return ctypes.CDLL(build.AMGE_SO)


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amge_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared("amge.h")
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
    from paper_2107_05613_gb300 import build

    out = subprocess.run(["nm", "-D", "--defined-only", build.AMGE_SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (amge_\w+)", out))
    assert set(names) <= exported


def test_validation_without_gpu(lib):
    lib.amge_upload_levels.restype = ctypes.c_int
    lib.amge_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p(1)
    assert lib.amge_upload_levels(None, None, ctypes.byref(out)) == 1      # AMGE_EINVAL
    assert out.value is None
    assert b"descriptor" in lib.amge_last_error()
    assert lib.amge_hier_info(None, None, None, None) == 1
    assert lib.amge_vcycle(None, None, None, 1, 0, None) == 1
    assert lib.amge_pcg_solve(None, None, None, 1, None, None, None) == 1
    assert lib.amge_wait_status(None, None, None) == 1
    lib.amge_hier_free(None)
    # problem-level setup: unknown flag bits are refused before any CUDA call
    from paper_2107_05613_gb300.amge import AMGE_HCURL, AMGE_SETUP_TARGETS, amge_problem

    for flags, ok in ((4, False), (AMGE_SETUP_TARGETS | 8, False)):
        p = amge_problem(AMGE_HCURL, 4, 0, None, None, 1, 1, flags)
        assert lib.amge_setup_upload(ctypes.byref(p), None, ctypes.byref(out)) == 1
        assert b"flags" in lib.amge_last_error()


def test_binding_names_match_abi():
    """The Python binding exposes the ABI's entry points under the same names."""
    import importlib

    from paper_2107_05613_gb300 import build

    if not os.path.exists(build.AMGE_SO):
        build.build_amge_lib()
    amge = importlib.import_module("paper_2107_05613_gb300.amge")
    for name in _declared("amge.h"):
        if name in ("amge_hier_free",):
            continue
        assert hasattr(amge, name), name


def test_binding_structs_match_header():
    """Every struct the header defines has a ctypes twin in the binding with the same
    fields, in the same order, of the same sizes -- so an added or reordered field in
    include/amge.h cannot silently shift the binding's layout."""
    import ctypes as ct
    import importlib

    amge = importlib.import_module("paper_2107_05613_gb300.amge")
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "amge.h")).read(), flags=re.S)
    sizes = {"int32_t": 4, "int64_t": 8, "double": 8}
    structs = re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S)
    assert len(structs) >= 5
    for body, name in structs:
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"(?:const\s+)?(\w+)\s*(\*?)\s*(\w+)$", decl)
            assert m, (name, decl)
            ctype, ptr, fname = m.groups()
            fields.append((fname, 8 if ptr else sizes[ctype]))
        py = getattr(amge, name)
        assert [f[0] for f in py._fields_] == [f[0] for f in fields], name
        for (fname, size), (_, pytype) in zip(fields, py._fields_):
            assert ct.sizeof(pytype) == size, (name, fname)
