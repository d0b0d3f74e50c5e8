"""FP64 brute-force oracle (test infrastructure; see the package docstring).

Definition (Section 3.2 problem statement; direct form Eq. (3)): for FP32
points p_j and query q widened exactly to FP64,
S(j, q) = sum over ascending k of (p_jk - q_k)^2, each operation rounded to
nearest with no fused multiply-add; j is a neighbour iff S <= fl64(R*R).
Output: CSR with per-query ascending ids and dist2 = (float)S.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


@dataclass
class CSR:
    offsets: np.ndarray   # int64, m+1
    ids: np.ndarray       # int32, nnz (ascending within each row)
    dist2: np.ndarray     # float32, nnz

    @property
    def m(self) -> int:
        return len(self.offsets) - 1

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def row(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.ids[a:b], self.dist2[a:b]

    def counts(self) -> np.ndarray:
        return np.diff(self.offsets)


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        f32p = ctypes.POINTER(ctypes.c_float)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.snn_oracle_dist2.argtypes = [f32p, f32p, i32]
        lib.snn_oracle_dist2.restype = f64
        lib.snn_oracle_count.argtypes = [f32p, i64, i32, i64, f32p, i64, i64, f64, i64p]
        lib.snn_oracle_count.restype = i64
        lib.snn_oracle_fill.argtypes = [f32p, i64, i32, i64, f32p, i64, i64, f64, i64p, i32p, f32p]
        lib.snn_oracle_fill.restype = None
        lib.snn_oracle_pairs.argtypes = [f32p, i32, i64, f32p, i64, i64p, i64p, i64, f64p]
        lib.snn_oracle_pairs.restype = None
        lib.snn_oracle_threads.argtypes = []
        lib.snn_oracle_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _as_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("expected a 2-d array")
    return a


def oracle_threads() -> int:
    return int(_get().snn_oracle_threads())


def brute_radius(P: np.ndarray, Q: np.ndarray | None, R: float) -> CSR:
    """All j with S(j, q) <= fl64(R*R) for every row q of Q (Q=None: Q=P)."""
    lib = _get()
    P = _as_f32(P)
    Q = P if Q is None else _as_f32(Q)
    if Q.shape[1] != P.shape[1]:
        raise ValueError("dimension mismatch")
    n, d = P.shape
    m = Q.shape[0]
    R2 = float(np.float64(R) * np.float64(R))
    counts = np.zeros(max(m, 1), dtype=np.int64)
    if m == 0 or n == 0:
        return CSR(np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    lib.snn_oracle_count(_ptr(P, ctypes.c_float), n, d, d, _ptr(Q, ctypes.c_float), m, d, R2,
                         _ptr(counts, ctypes.c_int64))
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts[:m], out=offsets[1:])
    nnz = int(offsets[-1])
    ids = np.empty(max(nnz, 1), dtype=np.int32)
    d2 = np.empty(max(nnz, 1), dtype=np.float32)
    lib.snn_oracle_fill(_ptr(P, ctypes.c_float), n, d, d, _ptr(Q, ctypes.c_float), m, d, R2,
                        _ptr(offsets, ctypes.c_int64), _ptr(ids, ctypes.c_int32),
                        _ptr(d2, ctypes.c_float))
    return CSR(offsets, ids[:nnz], d2[:nnz])


def brute_radius_numpy(P: np.ndarray, Q: np.ndarray | None, R: float) -> CSR:
    """The same definition in numpy (vectorised over pairs, ascending k,
    separate subtract / multiply / add: numpy never fuses them).  Small inputs."""
    P = np.asarray(P, dtype=np.float32).astype(np.float64)
    Q = P if Q is None else np.asarray(Q, dtype=np.float32).astype(np.float64)
    m, d = Q.shape
    R2 = np.float64(R) * np.float64(R)
    S = np.zeros((m, P.shape[0]), dtype=np.float64)
    for k in range(d):
        t = P[None, :, k] - Q[:, None, k]
        S = S + t * t
    mask = S <= R2
    counts = mask.sum(axis=1)
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    qi, pj = np.nonzero(mask)          # row-major: ascending j within each i
    return CSR(offsets, pj.astype(np.int32), S[qi, pj].astype(np.float32))


def pair_dist2(P: np.ndarray, Q: np.ndarray | None, qi: np.ndarray, pj: np.ndarray) -> np.ndarray:
    """S(pj[t], Q[qi[t]]) in FP64 for explicit pairs (Q=None: Q=P)."""
    lib = _get()
    P = _as_f32(P)
    Q = P if Q is None else _as_f32(Q)
    qi = np.ascontiguousarray(qi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    out = np.empty(len(qi), dtype=np.float64)
    if len(qi):
        lib.snn_oracle_pairs(_ptr(P, ctypes.c_float), P.shape[1], P.shape[1],
                             _ptr(Q, ctypes.c_float), Q.shape[1],
                             _ptr(qi, ctypes.c_int64), _ptr(pj, ctypes.c_int64), len(qi),
                             _ptr(out, ctypes.c_double))
    return out


def radius_rows(P: np.ndarray, Q: np.ndarray | None, rows: np.ndarray, R: float,
                margin: float = 1e-9) -> CSR:
    """The neighbour lists of the query rows ``rows`` of Q (Q=None: of P), by
    the definition of ``brute_radius``, for large P (sampled checks at full
    size).  Row t of the result belongs to query ``rows[t]``.

    A float64 matrix product gives G = ||p||^2 + ||q||^2 - 2 p.q.  In any
    summation order it is within gamma_{d+2} (||p||^2 + ||q||^2 + 2 sum |p_k
    q_k|) <= 2 gamma_{d+2} (||p||^2 + ||q||^2) of the exact ||p - q||^2
    (gamma_k = k u / (1 - k u), u = 2^-53), and the definition's S is within
    gamma_{d+2} ||p - q||^2 of it, so every pair with S <= fl64(R*R) has
    G <= R2 + margin (R2 + ||p||^2 + ||q||^2) whenever margin >= 4
    gamma_{d+2}.  Every pair inside that margin is then evaluated by the
    definition itself (``snn_oracle_pairs``: ascending k, FP64, no FMA) and
    decided by S <= R2; the product only discards pairs that are certainly
    outside."""
    P = _as_f32(P)
    Qs = _as_f32((P if Q is None else _as_f32(Q))[np.asarray(rows, dtype=np.int64)])
    n, d = P.shape
    if d < 64:
        # low d: the product costs more than the definition itself
        return brute_radius(P, Qs, R)
    u = 2.0 ** -53
    if not margin >= 4.0 * (d + 2) * u / (1.0 - (d + 2) * u):
        raise ValueError("margin below the rounding bound of the matrix product")
    R2 = float(np.float64(R) * np.float64(R))
    P64 = P.astype(np.float64)
    pn = np.einsum("ij,ij->i", P64, P64)
    m = Qs.shape[0]
    step = max(1, int(2e7 // max(n, 1)))
    qi_all, pj_all = [], []
    for a in range(0, m, step):
        Qc = Qs[a:a + step].astype(np.float64)
        qn = np.einsum("ij,ij->i", Qc, Qc)
        G = qn[:, None] + pn[None, :] - 2.0 * (Qc @ P64.T)
        mask = G <= R2 + margin * (R2 + qn[:, None] + pn[None, :])
        qi, pj = np.nonzero(mask)          # row-major: ascending j within a row
        qi_all.append(qi + a)
        pj_all.append(pj)
    qi = np.concatenate(qi_all) if qi_all else np.zeros(0, np.int64)
    pj = np.concatenate(pj_all) if pj_all else np.zeros(0, np.int64)
    S = pair_dist2(P, Qs, qi, pj)
    keep = S <= R2
    counts = np.bincount(qi[keep], minlength=m)
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return CSR(offsets, pj[keep].astype(np.int32), S[keep].astype(np.float32))


def radius_grid(P: np.ndarray, Q: np.ndarray | None, R: float, chunk: int = 8192) -> CSR:
    """The definition of ``brute_radius`` for every query, for large sets in
    low dimension (d <= 4): only pairs in the same or adjacent cells of a
    uniform grid of side h = R (1 + 1e-6) (1 for R = 0) are evaluated, by the
    definition itself (``snn_oracle_pairs``), and decided by S <= fl64(R*R).

    No neighbour is missed: S <= fl64(R*R) implies an exact distance of at
    most R (1 + 1e-15) (S is within gamma_{d+2} of it), hence every
    coordinate difference is below h, and the cells floor(x_k / h), computed
    in FP64 with |x_k / h| < 2^30, differ by at most one per axis."""
    P = _as_f32(P)
    Qa = P if Q is None else _as_f32(Q)
    n, d = P.shape
    m = Qa.shape[0]
    if d > 4:
        raise ValueError("radius_grid is for d <= 4")
    R2 = float(np.float64(R) * np.float64(R))
    # R = 0: only identical points (S = 0) are neighbours; any cell side works
    h = float(R) * (1.0 + 1e-6) if R > 0 else 1.0
    P64, Q64 = P.astype(np.float64), Qa.astype(np.float64)
    if max(np.abs(P64).max(initial=0.0), np.abs(Q64).max(initial=0.0)) / h >= 2.0 ** 30:
        raise ValueError("grid too fine for the coordinates")
    cp = np.floor(P64 / h).astype(np.int64)
    cq = np.floor(Q64 / h).astype(np.int64)
    lo = np.minimum(cp.min(axis=0, initial=0), cq.min(axis=0, initial=0)) - 1
    size = np.maximum(cp.max(axis=0, initial=0), cq.max(axis=0, initial=0)) - lo + 2
    radix = np.ones(d, dtype=np.int64)
    for k in range(1, d):
        radix[k] = radix[k - 1] * size[k - 1]
    if float(radix[-1]) * float(size[-1]) >= 2.0 ** 62:
        raise ValueError("grid too large")
    kp = ((cp - lo) * radix).sum(axis=1)
    kq = ((cq - lo) * radix).sum(axis=1)
    order = np.argsort(kp, kind="stable")
    ks = kp[order]
    shifts = np.array(np.meshgrid(*[[-1, 0, 1]] * d, indexing="ij")).reshape(d, -1).T
    offs = (shifts * radix).sum(axis=1)
    counts_all = np.zeros(m, dtype=np.int64)
    ids_parts, d2_parts = [], []
    for a in range(0, m, chunk):
        qk = kq[a:a + chunk]
        qis, pjs = [], []
        for o in offs:
            t = qk + o
            l = np.searchsorted(ks, t, side="left")
            r = np.searchsorted(ks, t, side="right")
            c = r - l
            tot = int(c.sum())
            if tot == 0:
                continue
            qi = np.repeat(np.arange(len(qk), dtype=np.int64), c)
            start = np.repeat(l - (np.cumsum(c) - c), c)
            pjs.append(order[start + np.arange(tot, dtype=np.int64)])
            qis.append(qi + a)
        if not qis:
            continue
        qi = np.concatenate(qis)
        pj = np.concatenate(pjs)
        S = pair_dist2(P, Qa, qi, pj)
        keep = S <= R2
        qi, pj, S = qi[keep], pj[keep], S[keep]
        srt = np.lexsort((pj, qi))
        qi, pj, S = qi[srt], pj[srt], S[srt]
        counts_all[a:a + chunk] = np.bincount(qi - a, minlength=len(qk))
        ids_parts.append(pj.astype(np.int32))
        d2_parts.append(S.astype(np.float32))
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts_all, out=offsets[1:])
    ids = np.concatenate(ids_parts) if ids_parts else np.zeros(0, np.int32)
    d2 = np.concatenate(d2_parts) if d2_parts else np.zeros(0, np.float32)
    return CSR(offsets, ids, d2)


def brute_row(P: np.ndarray, q: np.ndarray, R: float):
    """One query row against all of P: (ascending ids, dist2 float32)."""
    csr = brute_radius(P, np.asarray(q, dtype=np.float32).reshape(1, -1), R)
    return csr.row(0)
