"""Cosine and angular radius search by the Euclidean reduction of Section 3.

TEST INFRASTRUCTURE (see the package docstring): only tests, the smoke test
and the benchmark's CPU leg use it.

Section 3 reduces both measures to the Euclidean distance of normalised rows:
for unit vectors u, v the cosine distance is 1 - u.v = ||u - v||^2 / 2, and
the angle between them is at most alpha exactly when
||u - v||^2 <= 2 - 2 cos(alpha).

Reading of the rounding (the paper states the identities in exact
arithmetic):

* a row x becomes u_k = fl32(x_k * r) with r = 1 / sqrt(s) and
  s = sum over ascending k of x_k^2, all in FP64 with each operation
  rounded to nearest and no fused multiply-add (square root and division
  correctly rounded); a row of zeros stays zero;
* the search radius for a cosine-distance bound c is R = sqrt(2 c), for a
  cosine-similarity bound t (t = cos(alpha) for an angle bound alpha) it is
  R = sqrt(2 - 2 t), both in FP64;
* the neighbours are then exactly those of the Euclidean definition
  (``brute_radius``) on the normalised rows, with dist2 their squared
  Euclidean distance (twice the cosine distance).
"""
from __future__ import annotations

import math

import numpy as np

from .brute import CSR, brute_radius


def normalize_rows(X: np.ndarray) -> np.ndarray:
    """Unit rows by the reading above (FP32 in, FP32 out)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Xd = X.astype(np.float64)
    s = np.zeros(X.shape[0], dtype=np.float64)
    for k in range(X.shape[1]):          # ascending k, one rounding per step
        s = s + Xd[:, k] * Xd[:, k]
    out = np.zeros_like(X)
    nz = s > 0.0
    r = 1.0 / np.sqrt(s[nz])
    out[nz] = (Xd[nz] * r[:, None]).astype(np.float32)
    return out


def radius_for_cosine_distance(c: float) -> float:
    """R with R^2 = 2 c (cosine distance at most c)."""
    return math.sqrt(2.0 * float(c))


def radius_for_cosine_similarity(t: float) -> float:
    """R with R^2 = 2 - 2 t (cosine similarity at least t; t = cos(alpha))."""
    return math.sqrt(2.0 - 2.0 * float(t))


def cosine_radius(P: np.ndarray, Q: np.ndarray | None, R: float) -> CSR:
    """Neighbours of the normalised queries among the normalised points within
    Euclidean radius R (self-join when Q is None)."""
    return brute_radius(normalize_rows(P), None if Q is None else normalize_rows(Q), R)
