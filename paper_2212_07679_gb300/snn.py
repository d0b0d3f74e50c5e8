"""Thin ctypes binding of libsnn (include/snn.h).

Argument marshalling only: every step of the search runs in the CUDA library.
PyTorch supplies device memory and the current stream.  Importing this
module loads ``_build/libsnn.so`` and raises if it is missing or cannot be
loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsnn.so")

SNN_OK, SNN_EINVAL, SNN_ENOMEM, SNN_ECUDA, SNN_ETIMEOUT, SNN_EOVERFLOW, SNN_ENOTSUP = range(7)
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2}


class SNNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"snn status {status}: {msg}")
        self.status = status


class CSRStruct(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("offsets", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("dist2", ctypes.c_void_p)]


class StatsStruct(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("band_pairs", ctypes.c_int64),
                ("survivors", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("exact_fp64", ctypes.c_int64), ("mma_flops_per_pair", ctypes.c_int64),
                ("ms_prep", ctypes.c_float), ("ms_score", ctypes.c_float),
                ("ms_recheck", ctypes.c_float), ("ms_csr", ctypes.c_float),
                ("precision_used", ctypes.c_int32), ("split_used", ctypes.c_int32),
                ("ms_score_kernel", ctypes.c_float), ("flags", ctypes.c_int32)]

SNN_STATS_NO_CANDIDATES = 1


def _stats_struct(stats):
    """stats: False (none), True (every counter) or "phases" (no candidate
    count: SNN_STATS_NO_CANDIDATES, candidates = -1)."""
    if not stats:
        return None
    if stats not in (True, "phases"):
        raise ValueError("stats must be False, True or 'phases'")
    st = StatsStruct()
    if stats == "phases":
        st.flags = SNN_STATS_NO_CANDIDATES
    return st


class IPStatsStruct(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_double), ("radius", ctypes.c_double), ("band_pairs", ctypes.c_int64),
                ("survivors", ctypes.c_int64), ("candidates", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("exact_fp64", ctypes.c_int64)]


class ViewStruct(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("dp", ctypes.c_int32),
                ("mu", ctypes.c_void_p), ("v1", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("order", ctypes.c_void_p), ("points", ctypes.c_void_p),
                ("alpha_err", ctypes.c_double), ("centre", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsnn is not built ({LIB_PATH} missing); run "
                          "paper_2212_07679_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.snn_index_build.argtypes = [vp, i64, i32, i64, vp, ctypes.POINTER(vp)]
    lib.snn_index_build.restype = ctypes.c_int
    lib.snn_query_radius.argtypes = [vp, vp, i64, i64, f64, ctypes.c_int, vp,
                                     ctypes.POINTER(CSRStruct), ctypes.POINTER(StatsStruct)]
    lib.snn_query_radius.restype = ctypes.c_int
    lib.snn_query_radius_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(i64), ctypes.POINTER(i64),
                                           ctypes.POINTER(f64), ctypes.c_int, vp,
                                           ctypes.POINTER(CSRStruct)]
    lib.snn_query_radius_batch.restype = ctypes.c_int
    lib.snn_dbscan.argtypes = [vp, i64, i32, i64, f64, i32, ctypes.c_int, vp, vp, vp]
    lib.snn_dbscan.restype = ctypes.c_int
    lib.snn_index_get_view.argtypes = [vp, ctypes.POINTER(ViewStruct)]
    lib.snn_index_get_view.restype = ctypes.c_int
    lib.snn_free.argtypes = [vp]
    lib.snn_free.restype = None
    lib.snn_index_free.argtypes = [vp]
    lib.snn_index_free.restype = None
    lib.snn_last_error.argtypes = []
    lib.snn_last_error.restype = ctypes.c_char_p
    lib.snn_version.argtypes = []
    lib.snn_version.restype = ctypes.c_char_p
    lib.snn_index_insert.argtypes = [vp, vp, i64, i64, vp]
    lib.snn_index_insert.restype = ctypes.c_int
    lib.snn_index_delete.argtypes = [vp, vp, i64, vp]
    lib.snn_index_delete.restype = ctypes.c_int
    lib.snn_index_size.argtypes = [vp]
    lib.snn_index_size.restype = i64
    lib.snn_query_radius_each.argtypes = [vp, vp, i64, i64, vp, ctypes.c_int, vp,
                                          ctypes.POINTER(CSRStruct), ctypes.POINTER(StatsStruct)]
    lib.snn_query_radius_each.restype = ctypes.c_int
    lib.snn_inner_product_search.argtypes = [vp, i64, i32, i64, vp, i64, i64, f64, ctypes.c_int, vp,
                                             ctypes.POINTER(CSRStruct), ctypes.POINTER(IPStatsStruct)]
    lib.snn_inner_product_search.restype = ctypes.c_int
    lib.snn_normalize_rows.argtypes = [vp, i64, i32, i64, vp, i64, vp]
    lib.snn_normalize_rows.restype = ctypes.c_int
    lib.snn_radius_for_cosine_distance.argtypes = [f64]
    lib.snn_radius_for_cosine_distance.restype = f64
    lib.snn_radius_for_cosine_similarity.argtypes = [f64]
    lib.snn_radius_for_cosine_similarity.restype = f64
    lib.snn_test_inject.argtypes = [ctypes.c_int32]
    lib.snn_test_inject.restype = ctypes.c_int
    lib.snn_launch_count.argtypes = []
    lib.snn_launch_count.restype = ctypes.c_uint64
    lib.snn_index_saved_size.argtypes = [vp, ctypes.POINTER(i64)]
    lib.snn_index_saved_size.restype = ctypes.c_int
    lib.snn_index_save.argtypes = [vp, ctypes.c_char_p, i64, vp]
    lib.snn_index_save.restype = ctypes.c_int
    lib.snn_index_load.argtypes = [ctypes.c_char_p, i64, vp, ctypes.POINTER(vp)]
    lib.snn_index_load.restype = ctypes.c_int
    lib.snn_index_build_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                          ctypes.POINTER(i32), ctypes.POINTER(i64), vp,
                                          ctypes.POINTER(vp)]
    lib.snn_index_build_batch.restype = ctypes.c_int
    lib.snn_batch_plan_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                          ctypes.POINTER(f64), ctypes.c_int, i64, i64, vp,
                                          ctypes.POINTER(vp)]
    lib.snn_batch_plan_create.restype = ctypes.c_int
    lib.snn_batch_plan_queries.argtypes = [vp, i32]
    lib.snn_batch_plan_queries.restype = vp
    lib.snn_batch_plan_set_queries.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64), vp]
    lib.snn_batch_plan_set_queries.restype = ctypes.c_int
    lib.snn_batch_plan_run.argtypes = [vp, vp]
    lib.snn_batch_plan_run.restype = ctypes.c_int
    lib.snn_batch_plan_launch_graph.argtypes = [vp, vp]
    lib.snn_batch_plan_launch_graph.restype = ctypes.c_int
    lib.snn_batch_plan_result.argtypes = [vp, vp, ctypes.POINTER(CSRStruct), ctypes.POINTER(i64),
                                          ctypes.POINTER(i64)]
    lib.snn_batch_plan_result.restype = ctypes.c_int
    lib.snn_batch_plan_tune.argtypes = [vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                        ctypes.POINTER(ctypes.c_float)]
    lib.snn_batch_plan_tune.restype = ctypes.c_int
    lib.snn_batch_plan_config.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                          ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i32)]
    lib.snn_batch_plan_config.restype = ctypes.c_int
    lib.snn_batch_plan_free.argtypes = [vp, vp]
    lib.snn_batch_plan_free.restype = None
    return lib


lib = _load()


def _check(status: int):
    if status != SNN_OK:
        raise SNNError(status, lib.snn_last_error().decode(errors="replace"))


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _points(X: torch.Tensor, name: str):
    if not isinstance(X, torch.Tensor) or not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2:
        raise TypeError(f"{name} must be a 2-d float32 CUDA tensor")
    if X.stride(1) != 1:
        X = X.contiguous()
    return X, X.stride(0)


class _DeviceBuffer:
    """Library-allocated device memory exposed to torch; freed with snn_free."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.ptr = ptr
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}

    def __del__(self):
        if self.ptr:
            lib.snn_free(ctypes.c_void_p(self.ptr))
            self.ptr = 0


def _wrap(ptr: int, count: int, typestr: str, dtype, device) -> torch.Tensor:
    if not ptr or count == 0:
        if ptr:
            lib.snn_free(ctypes.c_void_p(ptr))
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_DeviceBuffer(ptr, count, typestr), device=device)


@dataclass
class CSR:
    """Neighbour lists: row r is indices[offsets[r]:offsets[r+1]] (original
    point ids, ascending) with dist2 the matching squared distances."""
    offsets: torch.Tensor
    indices: torch.Tensor
    dist2: torch.Tensor
    stats: dict | None = None

    @property
    def m(self) -> int:
        return self.offsets.numel() - 1

    @property
    def nnz(self) -> int:
        return self.indices.numel()

    def to_host(self, buffers: "HostBuffers | None" = None, stream=None, blocking: bool = True) -> "CSR":
        """Copies the lists into pinned host memory (reused from `buffers` when
        given) with asynchronous copies on `stream` (default: the current
        stream), then waits for them (blocking=False: returns at once; the
        host tensors are complete once `stream` has reached this point).
        Returns a CSR of host tensors."""
        b = buffers if buffers is not None else HostBuffers()
        off = b.take("offsets", self.offsets.numel(), torch.int64)
        idx = b.take("indices", self.indices.numel(), torch.int32)
        d2 = b.take("dist2", self.dist2.numel(), torch.float32)
        s = stream if stream is not None else torch.cuda.current_stream(self.offsets.device)
        with torch.cuda.stream(s):
            off.copy_(self.offsets, non_blocking=True)
            idx.copy_(self.indices, non_blocking=True)
            d2.copy_(self.dist2, non_blocking=True)
        if blocking:
            s.synchronize()
        return CSR(off, idx, d2, self.stats)


class HostBuffers:
    """Pinned host storage for CSR.to_host, grown on demand and reused."""

    def __init__(self):
        self._bufs = {}

    def take(self, name: str, n: int, dtype) -> torch.Tensor:
        t = self._bufs.get(name)
        if t is None or t.numel() < n or t.dtype != dtype:
            t = torch.empty(max(1, n + n // 4), dtype=dtype, pin_memory=True)
            self._bufs[name] = t
        return t[:n]


def _csr_from(cs: CSRStruct, device, stats=None) -> CSR:
    off = _wrap(cs.offsets, cs.m + 1, "<i8", torch.int64, device)
    idx = _wrap(cs.indices, cs.nnz, "<i4", torch.int32, device)
    d2 = _wrap(cs.dist2, cs.nnz, "<f4", torch.float32, device)
    return CSR(off, idx, d2, stats)


class Index:
    """SNN index (Algorithm 1) of the rows of a float32 CUDA tensor."""

    def __init__(self, X: torch.Tensor, stream=None):
        X, ld = _points(X, "X")
        self.device = X.device
        self.n, self.d = X.shape
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.snn_index_build(ctypes.c_void_p(X.data_ptr()), self.n, self.d, ld,
                                       _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def save(self, stream=None) -> bytes:
        """The index record as a byte image (snn_index_save): store it with
        open(path, "wb").write(...) and restore it with Index.load."""
        if self._h is None:
            raise ValueError("index is closed")
        nb = ctypes.c_int64()
        _check(lib.snn_index_saved_size(self._h, ctypes.byref(nb)))
        buf = ctypes.create_string_buffer(nb.value)
        with torch.cuda.device(self.device):
            _check(lib.snn_index_save(self._h, buf, nb.value, _stream_ptr(stream)))
        return buf.raw

    @classmethod
    def load(cls, image: bytes, device=None, stream=None) -> "Index":
        """An index from a byte image of Index.save (snn_index_load), on
        `device` (default: the current CUDA device)."""
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.snn_index_load(image, len(image), _stream_ptr(stream), ctypes.byref(h)))
        ix = cls.__new__(cls)
        ix.device = dev
        ix._h = h
        ix.n = int(lib.snn_index_size(h))
        ix.d = int.from_bytes(image[12:16], "little", signed=True)
        return ix

    def insert(self, X: torch.Tensor, stream=None) -> None:
        """Adds the rows of X as points n, n+1, ... (snn_index_insert)."""
        if self._h is None:
            raise ValueError("index is closed")
        X, ld = _points(X, "X")
        if X.shape[1] != self.d:
            raise ValueError(f"X must have {self.d} columns")
        with torch.cuda.device(self.device):
            _check(lib.snn_index_insert(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[0], ld,
                                        _stream_ptr(stream)))
        self.n = int(lib.snn_index_size(self._h))

    def delete(self, ids, stream=None) -> None:
        """Removes the listed point ids; the rest are renumbered 0, 1, ... in
        their previous order (snn_index_delete)."""
        if self._h is None:
            raise ValueError("index is closed")
        t = torch.as_tensor(ids, dtype=torch.int32, device=self.device).contiguous()
        with torch.cuda.device(self.device):
            _check(lib.snn_index_delete(self._h, ctypes.c_void_p(t.data_ptr()), t.numel(),
                                        _stream_ptr(stream)))
        self.n = int(lib.snn_index_size(self._h))

    def query(self, Q: torch.Tensor | None = None, R: float = 0.0, precision: str = "fp32",
              stats: bool | str = False, stream=None) -> CSR:
        """Algorithm 2 for all rows of Q (None: self-join).  stats: False,
        True (every counter) or "phases" (no candidate-range count)."""
        if self._h is None:
            raise RuntimeError("index was freed")
        cs = CSRStruct()
        st = _stats_struct(stats)
        if Q is None:
            qptr, m, ldq = None, 0, self.d
        else:
            Q, ldq = _points(Q, "Q")
            if Q.shape[1] != self.d:
                raise ValueError("Q has the wrong number of columns")
            if Q.shape[0] == 0:
                # an empty query set still needs a non-NULL pointer (NULL
                # selects the self-join)
                Q = torch.empty((1, self.d), dtype=torch.float32, device=self.device)
                qptr, m, ldq = ctypes.c_void_p(Q.data_ptr()), 0, self.d
            else:
                qptr, m = ctypes.c_void_p(Q.data_ptr()), Q.shape[0]
        with torch.cuda.device(self.device):
            _check(lib.snn_query_radius(self._h, qptr, m, ldq, float(R), PRECISIONS[precision],
                                        _stream_ptr(stream), ctypes.byref(cs),
                                        ctypes.byref(st) if st is not None else None))
        sd = None
        if st is not None:
            sd = {k: getattr(st, k) for k, _ in StatsStruct._fields_}
        return _csr_from(cs, self.device, sd)

    def query_each(self, Q: torch.Tensor, R, precision: str = "fp32", stats: bool | str = False,
                   stream=None) -> CSR:
        """Out-of-sample queries with one radius each (snn_query_radius_each);
        R: a float64 sequence or tensor of len(Q) radii."""
        if self._h is None:
            raise ValueError("index is closed")
        Q, ldq = _points(Q, "Q")
        Rt = torch.as_tensor(R, dtype=torch.float64, device=self.device).contiguous()
        if Rt.numel() != Q.shape[0]:
            raise ValueError("one radius per query row")
        cs = CSRStruct()
        st = _stats_struct(stats)
        with torch.cuda.device(self.device):
            _check(lib.snn_query_radius_each(self._h, ctypes.c_void_p(Q.data_ptr()), Q.shape[0], ldq,
                                             ctypes.c_void_p(Rt.data_ptr()), PRECISIONS[precision],
                                             _stream_ptr(stream), ctypes.byref(cs),
                                             ctypes.byref(st) if st is not None else None))
        sd = {k: getattr(st, k) for k, _ in StatsStruct._fields_} if st is not None else None
        return _csr_from(cs, self.device, sd)

    def view(self) -> dict:
        """Device arrays of the index (copies), for inspection and tests."""
        v = ViewStruct()
        _check(lib.snn_index_get_view(self._h, ctypes.byref(v)))
        n, d, dp = v.n, v.d, v.dp

        def cp(ptr, count, typestr, dtype):
            t = torch.as_tensor(_Borrowed(ptr, count, typestr), device=self.device)
            return t.clone()
        return {
            "mu": cp(v.mu, d, "<f8", torch.float64),
            "v1": cp(v.v1, d, "<f8", torch.float64),
            "alpha": cp(v.alpha, n, "<f4", torch.float32),
            "order": cp(v.order, n, "<i4", torch.int32),
            "points": cp(v.points, n * dp, "<f4", torch.float32).view(n, dp)[:, :d],
            "alpha_err": v.alpha_err,
            "centre": cp(v.centre, d, "<f4", torch.float32),
        }

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.snn_index_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Borrowed:
    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def radius_search(X: torch.Tensor, Q: torch.Tensor | None, R: float, precision: str = "fp32",
                  stats: bool = False) -> CSR:
    """Index X and query every row of Q (None: self-join)."""
    return Index(X).query(Q, R, precision, stats)


def normalize_rows(X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Unit rows for cosine / angular search (Section 3): u = fl32(x r),
    r = 1 / sqrt(sum of x_k^2) in FP64 (see snn_normalize_rows)."""
    X, ld = _points(X, "X")
    if out is None:
        out = torch.empty_like(X)
    o, ldo = _points(out, "out")
    if o.shape != X.shape:
        raise ValueError("out must have the shape of X")
    with torch.cuda.device(X.device):
        _check(lib.snn_normalize_rows(ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], ld,
                                      ctypes.c_void_p(o.data_ptr()), ldo, _stream_ptr(stream)))
    return o


def radius_for_cosine_distance(c: float) -> float:
    """Euclidean radius on unit rows for cosine distance <= c: sqrt(2 c)."""
    r = lib.snn_radius_for_cosine_distance(float(c))
    if r != r:
        raise ValueError("cosine distance bound must lie in [0, 2]")
    return r


def radius_for_cosine_similarity(t: float) -> float:
    """Euclidean radius on unit rows for cosine similarity >= t (an angle
    bound alpha: t = cos(alpha)): sqrt(2 - 2 t)."""
    r = lib.snn_radius_for_cosine_similarity(float(t))
    if r != r:
        raise ValueError("cosine similarity bound must lie in [-1, 1]")
    return r


def cosine_radius_search(X: torch.Tensor, Q: torch.Tensor | None = None, *,
                         cos_sim: float | None = None, cos_dist: float | None = None,
                         precision: str = "bf16", stats: bool = False, stream=None) -> CSR:
    """All rows of X within a cosine similarity (>= cos_sim) or cosine
    distance (<= cos_dist) bound of each row of Q (None: self-join), by the
    Euclidean search on normalised rows; dist2 is twice the cosine distance
    of the normalised rows."""
    if (cos_sim is None) == (cos_dist is None):
        raise ValueError("give exactly one of cos_sim and cos_dist")
    R = (radius_for_cosine_similarity(cos_sim) if cos_sim is not None
         else radius_for_cosine_distance(cos_dist))
    U = normalize_rows(X, stream=stream)
    V = None if Q is None else normalize_rows(Q, stream=stream)
    return Index(U, stream=stream).query(V, R, precision, stats, stream=stream)


def inner_product_search(P: torch.Tensor, Q: torch.Tensor, tau: float, precision: str = "bf16",
                         stats: bool = False, stream=None) -> CSR:
    """Every row of P whose FP64 dot product with a row of Q reaches tau
    (snn_inner_product_search); the CSR's dist2 holds the dot products."""
    P, ldp = _points(P, "P")
    Q, ldq = _points(Q, "Q")
    if P.shape[1] != Q.shape[1]:
        raise ValueError("P and Q must have the same number of columns")
    cs = CSRStruct()
    st = IPStatsStruct() if stats else None
    with torch.cuda.device(P.device):
        _check(lib.snn_inner_product_search(ctypes.c_void_p(P.data_ptr()), P.shape[0], P.shape[1], ldp,
                                            ctypes.c_void_p(Q.data_ptr()), Q.shape[0], ldq, float(tau),
                                            PRECISIONS[precision], _stream_ptr(stream), ctypes.byref(cs),
                                            ctypes.byref(st) if st is not None else None))
    sd = {k: getattr(st, k) for k, _ in IPStatsStruct._fields_} if st is not None else None
    return _csr_from(cs, P.device, sd)


def query_batch(indices: list[Index], Qs: list[torch.Tensor | None], Rs: list[float],
                precision: str = "fp32", stream=None) -> list[CSR]:
    """Many independent (index, queries, radius) problems in one library call."""
    k = len(indices)
    hs = (ctypes.c_void_p * k)(*[ix.handle.value for ix in indices])
    qp = (ctypes.c_void_p * k)()
    ms = (ctypes.c_int64 * k)()
    lds = (ctypes.c_int64 * k)()
    keep = []
    for s, (ix, Q) in enumerate(zip(indices, Qs)):
        if Q is None:
            qp[s], ms[s], lds[s] = None, 0, ix.d
        else:
            Q, ld = _points(Q, "Q")
            if Q.shape[0] == 0:
                Q, ld = torch.empty((1, ix.d), dtype=torch.float32, device=ix.device), ix.d
                keep.append(Q)
                qp[s], ms[s], lds[s] = Q.data_ptr(), 0, ld
                continue
            keep.append(Q)
            qp[s], ms[s], lds[s] = Q.data_ptr(), Q.shape[0], ld
    rs = (ctypes.c_double * k)(*[float(r) for r in Rs])
    outs = (CSRStruct * k)()
    dev = indices[0].device if k else torch.device("cuda")
    with torch.cuda.device(dev):
        _check(lib.snn_query_radius_batch(k, hs, qp, ms, lds, rs, PRECISIONS[precision],
                                          _stream_ptr(stream), outs))
    return [_csr_from(outs[s], dev) for s in range(k)]


def build_batch(Xs: list, stream=None) -> list:
    """Indices of many small point sets (d <= 64) built together
    (snn_index_build_batch): one launch per step over every set."""
    k = len(Xs)
    pts = [_points(X, "X") for X in Xs]
    xp = (ctypes.c_void_p * k)(*[X.data_ptr() for X, _ in pts])
    ns = (ctypes.c_int64 * k)(*[X.shape[0] for X, _ in pts])
    ds = (ctypes.c_int32 * k)(*[X.shape[1] for X, _ in pts])
    lds = (ctypes.c_int64 * k)(*[ld for _, ld in pts])
    hs = (ctypes.c_void_p * k)()
    dev = pts[0][0].device if k else torch.device("cuda")
    with torch.cuda.device(dev):
        _check(lib.snn_index_build_batch(k, xp, ns, ds, lds, _stream_ptr(stream), hs))
    out = []
    for t, (X, _) in enumerate(pts):
        ix = Index.__new__(Index)
        ix.device = dev
        ix.n, ix.d = X.shape
        ix._h = ctypes.c_void_p(hs[t])
        out.append(ix)
    return out


class _PlanViews:
    """Per-set CSR views of a batch plan's result arrays: the sets' arrays are
    slices of three plan arrays, each wrapped once as a tensor over its span
    and narrowed per set on access."""

    _ARRAYS = (("offsets", 8, "<i8", torch.int64), ("indices", 4, "<i4", torch.int32),
               ("dist2", 4, "<f4", torch.float32))

    def __init__(self, outs, device):
        self._outs = outs
        self._device = device
        self._spans = {}
        for key, size, typestr, dtype in self._ARRAYS:
            ext = [(getattr(c, key), self._count(c, key)) for c in outs]
            ext = [(p, n) for p, n in ext if p and n > 0]
            if ext:
                lo = min(p for p, _ in ext)
                hi = max(p + n * size for p, n in ext)
                self._spans[key] = (lo, size, torch.as_tensor(_Borrowed(lo, (hi - lo) // size, typestr),
                                                              device=device))

    @staticmethod
    def _count(c, key):
        return c.m + 1 if key == "offsets" else c.nnz

    def __len__(self):
        return len(self._outs)

    def __getitem__(self, t):
        if isinstance(t, slice):
            return [self[i] for i in range(*t.indices(len(self)))]
        if t < 0:
            t += len(self)
        c = self._outs[t]
        arrs = []
        for key, _, _, dtype in self._ARRAYS:
            ptr, n = getattr(c, key), self._count(c, key)
            if not ptr or n == 0:
                arrs.append(torch.empty(0, dtype=dtype, device=self._device))
            else:
                lo, size, base = self._spans[key]
                arrs.append(base.narrow(0, (ptr - lo) // size, n))
        return CSR(*arrs)

    def __iter__(self):
        return (self[t] for t in range(len(self)))


class BatchPlan:
    """A batched query with fixed sizes (snn_batch_plan_*): runs enqueue
    device work only, so they can be captured into a CUDA graph.  ms[t] is
    the number of queries of set t (written into queries(t) before a run), or
    None for the self-join of indices[t]."""

    def __init__(self, indices: list, ms: list, Rs: list, precision: str = "fp32",
                 survivor_capacity: int = 1 << 24, nnz_capacity: int = 1 << 24, stream=None):
        k = len(indices)
        self.indices = list(indices)          # the plan reads their arrays
        self.device = indices[0].device
        self.ms = [-1 if m is None else int(m) for m in ms]
        hs = (ctypes.c_void_p * k)(*[ix.handle.value for ix in indices])
        mm = (ctypes.c_int64 * k)(*self.ms)
        rs = (ctypes.c_double * k)(*[float(r) for r in Rs])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_create(k, hs, mm, rs, PRECISIONS[precision],
                                             int(survivor_capacity), int(nnz_capacity),
                                             _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def queries(self, t: int) -> torch.Tensor:
        """The plan's device buffer for set t's queries (m x d), writable."""
        p = lib.snn_batch_plan_queries(self._h, t)
        if not p or self.ms[t] <= 0:
            return torch.empty((0, self.indices[t].d), dtype=torch.float32, device=self.device)
        m, d = self.ms[t], self.indices[t].d
        return torch.as_tensor(_Borrowed(p, m * d, "<f4"), device=self.device).view(m, d)

    def set_queries(self, Qs: list, stream=None):
        """Copies every out-of-sample set's queries (Qs[t]: m x d FP32 device
        rows; None for self-join sets) into the plan in one launch
        (snn_batch_plan_set_queries)."""
        k = len(self.ms)
        if len(Qs) != k:
            raise ValueError("one query tensor (or None) per set")
        ptrs, lds, keep = [], [], []
        for t, q in enumerate(Qs):
            if self.ms[t] <= 0 or q is None:
                ptrs.append(None)
                lds.append(0)
                continue
            q, ld = _points(q, "Q")
            if q.shape != (self.ms[t], self.indices[t].d):
                raise ValueError(f"set {t}: queries must be {self.ms[t]} x {self.indices[t].d}")
            keep.append(q)
            ptrs.append(q.data_ptr())
            lds.append(ld)
        qp = (ctypes.c_void_p * k)(*ptrs)
        lp = (ctypes.c_int64 * k)(*lds)
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_set_queries(self._h, qp, lp, _stream_ptr(stream)))

    def run(self, stream=None):
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_run(self._h, _stream_ptr(stream)))

    def launch_graph(self, stream=None):
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_launch_graph(self._h, _stream_ptr(stream)))

    def tune(self, stream=None):
        c, t, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_tune(self._h, _stream_ptr(stream), ctypes.byref(c),
                                           ctypes.byref(t), ctypes.byref(ms)))
        return c.value, t.value, ms.value

    def config(self) -> dict:
        """Current scoring configuration: FP32 chunks per item and CTAs per SM,
        tensor-core groups and the mask of those scoring on the tensor cores,
        and whether the last tune() came from the tuning cache."""
        c, t, g, fc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        m = ctypes.c_uint32()
        _check(lib.snn_batch_plan_config(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(g),
                                         ctypes.byref(m), ctypes.byref(fc)))
        return {"chunks_per_item": c.value, "ctas_per_sm": t.value, "tc_groups": g.value,
                "tc_mask": m.value, "from_cache": bool(fc.value)}

    def result(self, stream=None, copy: bool = True):
        """Per-set results of the last run: a list of copies, or with
        copy=False a sequence of per-set views of the plan's arrays (made on
        access; valid until the next run)."""
        k = len(self.indices)
        outs = (CSRStruct * k)()
        ns, nz = ctypes.c_int64(), ctypes.c_int64()
        with torch.cuda.device(self.device):
            _check(lib.snn_batch_plan_result(self._h, _stream_ptr(stream), outs, ctypes.byref(ns),
                                             ctypes.byref(nz)))
        views = _PlanViews(outs, self.device)
        if not copy:
            return views
        return [CSR(v.offsets.clone(), v.indices.clone(), v.dist2.clone()) for v in views]

    def close(self, stream=None):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.snn_batch_plan_free(self._h, _stream_ptr(stream))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dbscan(X: torch.Tensor, eps: float, min_pts: int, precision: str = "fp32", stream=None):
    """DBSCAN with SNN neighbourhoods: (labels int32, is_core uint8)."""
    X, ld = _points(X, "X")
    n, d = X.shape
    labels = torch.empty(n, dtype=torch.int32, device=X.device)
    core = torch.empty(n, dtype=torch.uint8, device=X.device)
    with torch.cuda.device(X.device):
        _check(lib.snn_dbscan(ctypes.c_void_p(X.data_ptr()), n, d, ld, float(eps), int(min_pts),
                              PRECISIONS[precision], _stream_ptr(stream),
                              ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(core.data_ptr())))
    return labels, core


def version() -> str:
    return lib.snn_version().decode()


SNN_SPLIT_NONE, SNN_SPLIT_BF16X2, SNN_SPLIT_BF16X3, SNN_SPLIT_FP16X2, SNN_SPLIT_FP16X1, SNN_SPLIT_E4M3 = (
    0, 1, 2, 3, 4, 10)
SNN_FAULT_STALL_TC_PRODUCER = 1
SNN_FAULT_SMALL_SURVIVOR_BUFFER = 2
SNN_FAULT_DEVICE_ALLOC = 3


def test_inject(fault: int) -> None:
    """Arms a one-shot test fault (see snn_test_inject in include/snn.h)."""
    _check(lib.snn_test_inject(int(fault)))


def launch_count() -> int:
    """Kernels launched by libsnn in this process so far."""
    return int(lib.snn_launch_count())
