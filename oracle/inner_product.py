"""Inner-product threshold search (the maximum-inner-product variant of
Section 3).

TEST INFRASTRUCTURE (see the package docstring).

Definition: for FP32 points p_j and queries q widened exactly to FP64,
D(j, q) = sum over ascending k of p_jk * q_k, each product and sum rounded to
nearest in FP64 with no fused multiply-add (the products of FP32 values are
exact in FP64); j is returned for q iff D(j, q) >= tau.  Output: CSR with
per-query ascending ids and values fl32(D).

Section 3 reaches such points through the Euclidean distance of augmented
vectors: with xi = max_j ||p_j||, p~ = [sqrt(xi^2 - ||p||^2), p] and
q~ = [0, q], ||p~ - q~||^2 = xi^2 + ||q||^2 - 2 p.q.  That identity only
prunes; this module is the plain definition above.
"""
from __future__ import annotations

import numpy as np

from .brute import CSR


def dot_fp64(P: np.ndarray, q: np.ndarray) -> np.ndarray:
    """D(j, q) for every row of P by the definition (ascending k, FP64)."""
    P = np.asarray(P, dtype=np.float32).astype(np.float64)
    q = np.asarray(q, dtype=np.float32).astype(np.float64)
    D = np.zeros(P.shape[0], dtype=np.float64)
    for k in range(P.shape[1]):
        D = D + P[:, k] * q[k]
    return D


def brute_inner_product(P: np.ndarray, Q: np.ndarray, tau: float) -> CSR:
    """All (query, point) pairs with D >= tau, as CSR over the queries."""
    P = np.ascontiguousarray(P, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    offs = [0]
    ids, vals = [], []
    for i in range(Q.shape[0]):
        D = dot_fp64(P, Q[i])
        j = np.nonzero(D >= tau)[0]
        ids.append(j.astype(np.int32))
        vals.append(D[j].astype(np.float32))
        offs.append(offs[-1] + len(j))
    return CSR(np.asarray(offs, dtype=np.int64),
               np.concatenate(ids) if ids else np.zeros(0, np.int32),
               np.concatenate(vals) if vals else np.zeros(0, np.float32))
