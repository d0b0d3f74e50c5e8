"""Builds libsnn.so in-tree with nvcc for sm_103a (no cmake, no torch).

Every .cu under csrc/ is compiled to an object in parallel, then linked into
paper_2212_07679_gb300/_build/libsnn.so.  Objects are rebuilt when their
source, a header, or the flags change.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsnn.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in [shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsnn")


def _digest(paths, extra):
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()[:16]


def _compile(src, obj, extra):
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    return r.stderr


def build(verbose: bool = False, extra: list[str] | None = None, jobs: int | None = None) -> str:
    extra = list(extra or [])
    os.makedirs(OUT, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_digest = _digest(headers, extra + ARCH + FLAGS)
    objs, todo = [], []
    for src in srcs:
        tag = _digest([src], [hdr_digest])
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + f".{tag}.o")
        objs.append(obj)
        if not os.path.exists(obj):
            todo.append((src, obj))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(8, len(todo))) as ex:
            futs = {ex.submit(_compile, s, o, extra): s for s, o in todo}
            for f in cf.as_completed(futs):
                msg = f.result()
                if verbose and msg:
                    print(msg)
    link_tag = _digest(objs, [])
    stamp = LIB + ".stamp"
    if todo or not os.path.exists(LIB) or not os.path.exists(stamp) or open(stamp).read() != link_tag:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(link_tag)
    # drop objects of older source versions
    keep = set(objs)
    for o in glob.glob(os.path.join(OUT, "*.o")):
        if o not in keep:
            os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
