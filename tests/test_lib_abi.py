"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every function that include/snn.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2212_07679_gb300 import build as snn_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(snn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return snn_build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["snn_index_build", "snn_query_radius", "snn_query_radius_batch",
                     "snn_dbscan", "snn_free", "snn_index_free", "snn_last_error"]:
        assert required in names


def test_library_loads_and_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.snn_version.restype = ctypes.c_char_p
    lib.snn_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.snn_version()
    assert isinstance(lib.snn_last_error(), bytes)


def test_argument_validation_needs_no_gpu(libpath):
    # invalid arguments are rejected on the host before any CUDA call
    lib = ctypes.CDLL(libpath)
    lib.snn_index_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    assert lib.snn_index_build(None, 10, 3, 3, None, ctypes.byref(out)) == 1        # X NULL
    assert lib.snn_index_build(ctypes.c_void_p(16), 0, 3, 3, None, ctypes.byref(out)) == 1
    assert lib.snn_index_build(ctypes.c_void_p(16), 10, 0, 3, None, ctypes.byref(out)) == 1
    assert lib.snn_index_build(ctypes.c_void_p(16), 10, 5000, 5000, None, ctypes.byref(out)) == 1
    assert lib.snn_index_build(ctypes.c_void_p(16), 10, 4, 3, None, ctypes.byref(out)) == 1
    lib.snn_query_radius.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.snn_query_radius(None, None, 0, 0, 1.0, 0, None, None, None) == 1
    lib.snn_dbscan.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_double, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]
    assert lib.snn_dbscan(ctypes.c_void_p(16), 10, 3, 3, -1.0, 5, 0, None,
                          ctypes.c_void_p(16), ctypes.c_void_p(16)) == 1
    assert lib.snn_dbscan(ctypes.c_void_p(16), 10, 3, 3, 1.0, 0, 0, None,
                          ctypes.c_void_p(16), ctypes.c_void_p(16)) == 1
    lib.snn_free(None)
    lib.snn_index_free(None)


def test_fault_injection_arguments_need_no_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.snn_test_inject.argtypes = [ctypes.c_int32]
    assert lib.snn_test_inject(99) == 1
    assert lib.snn_test_inject(0) == 0
