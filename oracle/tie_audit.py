"""Exact-arithmetic audit of the FP64 definition's boundary decisions (test
infrastructure; see the package docstring).

The oracle decides "neighbour" by S <= fl64(R*R), with S the FP64 sum of
squared differences in ascending k (Section 3.2, Eq. (3)).  The paper's
problem asks for ||p - q|| <= R exactly.  The two differ only where rounding
moves S or R*R across the other.  This module finds every such pair.

FP32 inputs are integer multiples of 2^-149, so with P_k = p_k * 2^149 and
Q_k = q_k * 2^149 (Python integers) the exact squared distance is
E * 2^-298 with E = sum_k (P_k - Q_k)^2, and R (a double) is an exact
fraction.  Comparing E with R^2 * 2^298 therefore decides the exact question
with no rounding at all.

Only pairs near the boundary can flip.  Each difference, square and addition
of S rounds once, every term is non-negative, and FP32 data neither overflow
nor underflow in FP64, so |S - E'| <= gamma_{d+2} E' with E' the exact squared
distance and gamma_n = n u / (1 - n u), u = 2^-53; also
|fl64(R*R) - R^2| <= u R^2.  A flip therefore needs
|S - fl64(R*R)| <= 2 gamma_{d+2} S + 2 u fl64(R*R), and only pairs in that
band are evaluated exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_U = 2.0 ** -53


@dataclass
class AuditResult:
    band_pairs: int = 0                        # pairs evaluated exactly
    flips: list = field(default_factory=list)  # (query row, point id, S, exact_is_neighbour)

    @property
    def count(self) -> int:
        return len(self.flips)


def _scaled_int(x: float) -> int:
    # FP32 value x times 2^149: an integer, exactly representable as a double
    # (at most 2^277), so the conversion is exact
    return int(math.ldexp(float(x), 149))


def exact_is_neighbour(p: np.ndarray, q: np.ndarray, R: float) -> bool:
    """||p - q||^2 <= R^2 in exact rational arithmetic (p, q FP32 rows)."""
    e = 0
    for a, b in zip(p.astype(np.float32), q.astype(np.float32)):
        t = _scaled_int(a) - _scaled_int(b)
        e += t * t
    return Fraction(e) <= Fraction(float(R)) ** 2 * (1 << 298)


def fp64_dist2_block(P: np.ndarray, Qb: np.ndarray) -> np.ndarray:
    """S for every (query in Qb, point in P): the FP64 definition, ascending k,
    one rounding per difference, square and addition (numpy elementwise
    operations do not fuse)."""
    P64 = P.astype(np.float64)
    Q64 = Qb.astype(np.float64)
    S = np.zeros((Q64.shape[0], P64.shape[0]), dtype=np.float64)
    for k in range(P64.shape[1]):
        t = Q64[:, k, None] - P64[None, :, k]
        S = S + t * t
    return S


def tie_audit(P: np.ndarray, Q: np.ndarray | None, R: float, block: int = 64) -> AuditResult:
    """Pairs whose FP64 decision S <= fl64(R*R) differs from the exact one.

    P: n x d FP32 points; Q: m x d FP32 queries (None = the points themselves);
    R: the radius as a double.  Returns the number of boundary-band pairs that
    were evaluated exactly and the list of flips."""
    P = np.ascontiguousarray(P, dtype=np.float32)
    Q = P if Q is None else np.ascontiguousarray(Q, dtype=np.float32)
    d = P.shape[1]
    R = float(R)
    R2f = R * R
    nu = (d + 2) * _U
    gam = nu / (1.0 - nu)
    out = AuditResult()
    for a in range(0, Q.shape[0], block):
        S = fp64_dist2_block(P, Q[a:a + block])
        band = np.abs(S - R2f) <= 2.0 * gam * S + 2.0 * _U * R2f
        qi, pj = np.nonzero(band)
        out.band_pairs += len(qi)
        for i, j in zip(qi.tolist(), pj.tolist()):
            s = float(S[i, j])
            ex = exact_is_neighbour(P[j], Q[a + i], R)
            if ex != (s <= R2f):
                out.flips.append((a + i, j, s, ex))
    return out
