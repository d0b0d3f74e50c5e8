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
    assert lib.snn_test_inject(4) == 1
    for fault in (1, 2, 3):           # armed, then disarmed: no GPU call reaches them
        assert lib.snn_test_inject(fault) == 0
    assert lib.snn_test_inject(0) == 0


def test_cosine_radius_mappings_match_the_oracle(libpath):
    # host-only entry points: the FP64 radius of the Euclidean reduction
    import oracle
    lib = ctypes.CDLL(libpath)
    for fn in ("snn_radius_for_cosine_distance", "snn_radius_for_cosine_similarity"):
        getattr(lib, fn).argtypes = [ctypes.c_double]
        getattr(lib, fn).restype = ctypes.c_double
    for c in (0.0, 1e-9, 0.013, 0.5, 1.0, 1.75, 2.0):
        assert lib.snn_radius_for_cosine_distance(c) == oracle.radius_for_cosine_distance(c)
    for t in (-1.0, -0.3, 0.0, 0.5, 0.8660254037844387, 0.99, 1.0):
        assert lib.snn_radius_for_cosine_similarity(t) == oracle.radius_for_cosine_similarity(t)
    for bad in (-0.1, 2.5, float("nan")):
        r = lib.snn_radius_for_cosine_distance(bad)
        assert r != r
    r = lib.snn_radius_for_cosine_similarity(1.5)
    assert r != r


def test_normalize_rows_argument_validation_needs_no_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.snn_normalize_rows.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    p = ctypes.c_void_p(16)
    assert lib.snn_normalize_rows(None, 10, 3, 3, p, 3, None) == 1     # X NULL
    assert lib.snn_normalize_rows(p, 10, 3, 2, p, 3, None) == 1        # ld < d
    assert lib.snn_normalize_rows(p, 10, 3, 3, p, 2, None) == 1        # ldo < d
    assert lib.snn_normalize_rows(p, -1, 3, 3, p, 3, None) == 1        # n < 0
    assert lib.snn_normalize_rows(p, 0, 3, 3, p, 3, None) == 0         # nothing to do


def test_peak_probes_live_outside_the_search_library(libpath):
    # the roofline probes are a bench-only library linked against libsnn.so;
    # the search library itself does not export them
    import bench_probes
    assert not hasattr(ctypes.CDLL(libpath), "snn_measure_peak")
    lib = ctypes.CDLL(bench_probes.build())
    lib.snn_measure_peak.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    assert lib.snn_measure_peak(4, 1024, None, ctypes.byref(out)) == 1       # unknown kind
    assert lib.snn_measure_peak(-1, 1024, None, ctypes.byref(out)) == 1
    assert lib.snn_measure_peak(0, 63, None, ctypes.byref(out)) == 1         # iters < 64
    assert lib.snn_measure_peak(0, 1024, None, None) == 1                    # NULL output


def test_index_image_validation_needs_no_gpu(libpath):
    # a saved-index image is checked on the host before any device work
    import struct
    lib = ctypes.CDLL(libpath)
    lib.snn_index_load.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]
    lib.snn_index_saved_size.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    out = ctypes.c_void_p()
    nb = ctypes.c_int64()
    assert lib.snn_index_saved_size(None, ctypes.byref(nb)) == 1

    def header(magic=b"SNNIDX\x00\x01", version=1, d=8, n=100, dp=8):
        return magic + struct.pack("<iiqiiff", version, d, n, dp, 0, 0.0, 1.0)

    good = header()
    assert lib.snn_index_load(good[:20], 20, None, ctypes.byref(out)) == 1          # short header
    assert lib.snn_index_load(header(magic=b"NOTANIDX"), 40, None, ctypes.byref(out)) == 1
    assert lib.snn_index_load(header(version=2), 40, None, ctypes.byref(out)) == 1
    assert lib.snn_index_load(header(d=0, dp=0), 40, None, ctypes.byref(out)) == 1
    assert lib.snn_index_load(header(dp=12), 40, None, ctypes.byref(out)) == 1    # dp != roundup(d, 4)
    assert lib.snn_index_load(header(n=0), 40, None, ctypes.byref(out)) == 1
    assert lib.snn_index_load(good, len(good), None, ctypes.byref(out)) == 1      # arrays missing
    assert lib.snn_index_load(None, 0, None, ctypes.byref(out)) == 1
    assert out.value is None
