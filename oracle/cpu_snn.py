"""Plain CPU SNN in FP64: Algorithm 1 (index) and Algorithm 2 (query).

Test infrastructure (see the package docstring).  Steps follow the paper in
its order and notation, with numpy/LAPACK primitives as the steps:

Algorithm 1 (Section 3.1): mu = mean of the points; X = P - mu;
thin SVD X = U Sigma V^T (Eq. (1)); alpha_i = x_i^T v_1; sort so that
alpha_1 <= ... <= alpha_n; xbar_i = x_i^T x_i / 2.

Algorithm 2 (Section 3.2): x_q = q - mu; alpha_q = x_q^T v_1; candidate range
J = { j : |alpha_j - alpha_q| <= R } found by binary search (Eq. (2) makes
every neighbour a candidate); filter J.

Readings where the paper is silent:
* the window is widened by a bound on the FP64 rounding of alpha, so that no
  neighbour is lost to rounding (exact arithmetic needs no widening);
* the filter decides with the direct form Eq. (3) on the raw points, in the
  brute-force oracle's order, so the result equals the oracle's exactly.  The
  paper's filter Eq. (4) value, xbar_j - x_j^T x_q, is also returned for the
  analysis tests.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_U64 = 2.0 ** -53


@dataclass
class SNNIndex:
    mu: np.ndarray        # d, FP64
    X: np.ndarray         # n x d centred rows, sorted by alpha (FP64)
    P: np.ndarray         # n x d raw rows, sorted by alpha (FP32 values)
    v1: np.ndarray        # d, FP64, unit first principal direction
    alpha: np.ndarray     # n, sorted scores
    xbar: np.ndarray      # n, x_i^T x_i / 2
    order: np.ndarray     # n, original id of sorted position
    sigma: np.ndarray     # singular values of X
    eps: float            # bound on |computed alpha_i - exact alpha_i|


def snn_index(P: np.ndarray) -> SNNIndex:
    """Algorithm 1."""
    P = np.asarray(P, dtype=np.float32)
    n, d = P.shape
    P64 = P.astype(np.float64)
    mu = P64.mean(axis=0)
    X = P64 - mu[None, :]
    _, sigma, Vt = np.linalg.svd(X, full_matrices=False)
    v1 = Vt[0].copy()
    v1 /= np.linalg.norm(v1)
    alpha = X @ v1
    order = np.argsort(alpha, kind="stable")
    X = X[order]
    alpha = alpha[order]
    xbar = np.einsum("ij,ij->i", X, X) / 2.0
    # rounding of x = p - mu (u|x| per entry) and of the d-term dot product
    # (gamma_d sum |x_k v_k|), doubled for the norm of v1 and slack.
    eps = float(2.0 * (d + 3) * _U64 * np.max(np.abs(X) @ np.abs(v1))) if n else 0.0
    return SNNIndex(mu, X, P[order].copy(), v1, alpha, xbar, order, sigma, eps)


def snn_query(idx: SNNIndex, q: np.ndarray, R: float):
    """Algorithm 2 for one query.

    Returns (neighbour ids ascending, dist2 float32, candidate sorted range
    (lo, hi), Eq. (4) left-hand values over J).
    """
    q = np.asarray(q, dtype=np.float32)
    xq = q.astype(np.float64) - idx.mu
    aq = float(xq @ idx.v1)
    W = R * (1.0 + 2.0 ** -40) + 2.0 * idx.eps + 4.0 * _U64 * abs(aq)
    lo = int(np.searchsorted(idx.alpha, aq - W, side="left"))
    hi = int(np.searchsorted(idx.alpha, aq + W, side="right"))
    ip2 = idx.xbar[lo:hi] - idx.X[lo:hi] @ xq
    # direct form Eq. (3), ascending k, raw points (the oracle's definition)
    Pj = idx.P[lo:hi].astype(np.float64)
    qd = q.astype(np.float64)
    S = np.zeros(hi - lo, dtype=np.float64)
    for k in range(Pj.shape[1]):
        t = Pj[:, k] - qd[k]
        S = S + t * t
    keep = S <= np.float64(R) * np.float64(R)
    ids = idx.order[lo:hi][keep]
    d2 = S[keep].astype(np.float32)
    o = np.argsort(ids, kind="stable")
    return ids[o].astype(np.int32), d2[o], (lo, hi), ip2


def snn_radius(P: np.ndarray, Q: np.ndarray | None, R: float, idx: SNNIndex | None = None):
    """Index P (unless given) and query every row of Q (Q=None: Q=P).

    Returns (offsets, ids, dist2, candidates per query)."""
    idx = snn_index(P) if idx is None else idx
    Q = np.asarray(P if Q is None else Q, dtype=np.float32)
    offs = [0]
    ids_all, d2_all, cand = [], [], np.zeros(Q.shape[0], dtype=np.int64)
    for i in range(Q.shape[0]):
        ids, d2, (lo, hi), _ = snn_query(idx, Q[i], R)
        ids_all.append(ids)
        d2_all.append(d2)
        cand[i] = hi - lo
        offs.append(offs[-1] + len(ids))
    ids = np.concatenate(ids_all) if ids_all else np.zeros(0, np.int32)
    d2 = np.concatenate(d2_all) if d2_all else np.zeros(0, np.float32)
    return np.asarray(offs, dtype=np.int64), ids.astype(np.int32), d2.astype(np.float32), cand
