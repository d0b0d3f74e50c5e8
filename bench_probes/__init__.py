"""Bench-only throughput probes (tcgen05 BF16 / e4m3 MMAs, FP32 / FP64 FMAs).

``build()`` compiles peaks.cu into _build/libsnn_probes.so with nvcc for
sm_103a, linked against the search library (libsnn.so) for its error state
and launch helpers; ``measure_peak()`` runs one probe.  The search library
itself exports none of this.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsnn_probes.so")
KINDS = {"bf16_mma": 0, "e4m3_mma": 1, "fp32_fma": 2, "fp64_fma": 3}
_lib = None


def build() -> str:
    from paper_2212_07679_gb300 import build as snn_build
    snn_lib = snn_build.build()
    src = os.path.join(HERE, "peaks.cu")
    os.makedirs(OUT, exist_ok=True)
    deps = [src, os.path.join(HERE, "peaks.h"), snn_lib]
    if os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(p) for p in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = os.path.dirname(snn_lib)
    cmd = [snn_build.nvcc(), *snn_build.ARCH, *snn_build.FLAGS, "-I", HERE, "-shared", "-o", tmp, src,
           "-L", libdir, "-lsnn", "-lcudart", "-Xlinker", "-rpath=" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for peaks.cu:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _get():
    global _lib
    if _lib is None:
        from paper_2212_07679_gb300 import snn  # loads libsnn.so first
        lib = ctypes.CDLL(build())
        lib.snn_measure_peak.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double)]
        lib.snn_measure_peak.restype = ctypes.c_int
        _lib = (lib, snn)
    return _lib


def measure_peak(kind: str, iters: int, stream=None) -> float:
    """Rate (flop/s) of one arithmetic unit kept busy on every SM; see peaks.h."""
    lib, snn = _get()
    out = ctypes.c_double()
    snn._check(lib.snn_measure_peak(KINDS[kind], int(iters), snn._stream_ptr(stream), ctypes.byref(out)))
    return out.value
