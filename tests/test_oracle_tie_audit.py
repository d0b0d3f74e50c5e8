"""Pins of the exact-arithmetic tie audit (oracle/tie_audit.py): it finds a
planted pair that FP64 rounding moves inside the radius, it agrees with an
all-pairs rational brute force on data built to produce many such pairs, it
does not report exact ties, and on the seeded workloads the FP64 definition
and the exact question give the same neighbour sets (the count the
definition's rounding could change is zero)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2212_07679_gb300 import workloads as wl


def _rational_flips(P, Q, R):
    """All-pairs reference: exact squared distances as Fractions of the FP32
    values, against the FP64 definition's decisions from the numpy oracle."""
    csr = oracle.brute_radius_numpy(P, Q, R)
    flips = set()
    R2 = Fraction(float(R)) ** 2
    for i in range(Q.shape[0]):
        fp64_in = set(csr.row(i)[0].tolist())
        for j in range(P.shape[0]):
            e = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(P[j], Q[i]))
            if (e <= R2) != (j in fp64_in):
                flips.add((i, j))
    return flips


def test_planted_flip_is_found():
    # ||p - q||^2 = 2^40 + 2^-20 exactly; FP64 rounds the sum to 2^40 = R*R,
    # so the definition counts p as a neighbour and the exact question does not
    P = np.array([[2.0 ** 20, 2.0 ** -10]], dtype=np.float32)
    Q = np.zeros((1, 2), dtype=np.float32)
    R = 2.0 ** 20
    assert oracle.brute_radius_numpy(P, Q, R).nnz == 1
    res = oracle.tie_audit(P, Q, R)
    assert res.count == 1
    qi, pj, s, exact_in = res.flips[0]
    assert (qi, pj, s, exact_in) == (0, 0, 2.0 ** 40, False)
    assert not oracle.exact_is_neighbour(P[0], Q[0], R)


def test_audit_matches_rational_brute_force():
    # coordinates a * 2^20 and b * 2^-10 with small integers a, b: whenever the
    # large parts sit exactly on R the small parts are lost to rounding
    rng = np.random.default_rng(wl.SEED_BASE + 40)
    n, m = 48, 24
    P = np.stack([rng.integers(0, 4, n) * 2.0 ** 20, rng.integers(0, 4, n) * 2.0 ** -10,
                  rng.integers(0, 2, n) * 2.0 ** 19], axis=1).astype(np.float32)
    Q = np.stack([rng.integers(0, 4, m) * 2.0 ** 20, rng.integers(0, 4, m) * 2.0 ** -10,
                  rng.integers(0, 2, m) * 2.0 ** 19], axis=1).astype(np.float32)
    R = 2.0 ** 21
    ref = _rational_flips(P, Q, R)
    res = oracle.tie_audit(P, Q, R, block=7)
    assert len(ref) > 10
    assert {(i, j) for i, j, _, _ in res.flips} == ref
    assert all(not ex for _, _, _, ex in res.flips)        # FP64 includes, exact excludes
    assert res.band_pairs >= len(ref)


def test_random_small_data_matches_rational_brute_force():
    rng = np.random.default_rng(wl.SEED_BASE + 41)
    P = rng.standard_normal((40, 5)).astype(np.float32)
    Q = rng.standard_normal((12, 5)).astype(np.float32)
    # a radius exactly on one pair's FP64 distance puts that pair in the band
    R = float(np.sqrt(np.sum((P[3].astype(np.float64) - Q[2]) ** 2)))
    ref = _rational_flips(P, Q, R)
    res = oracle.tie_audit(P, Q, R)
    assert res.band_pairs >= 1
    assert {(i, j) for i, j, _, _ in res.flips} == ref


def test_exact_ties_are_not_flips():
    # 3-4-5 right triangles: every distance is exact, several equal R
    P = np.array([[0, 0], [3, 4], [-3, 4], [3, -4], [5, 0], [1, 1]], dtype=np.float32)
    res = oracle.tie_audit(P, None, 5.0)
    assert res.band_pairs >= 8          # the eight ordered pairs at distance exactly 5
    assert res.count == 0


@pytest.mark.parametrize("name,rows", [("gmm_iso", None), ("gmm_aniso", 48), ("lowrank_img", 12),
                                       ("blobs3d", 64)])
def test_seeded_workloads_have_no_flips(name, rows):
    w = wl.by_name(name)
    if rows is None:
        P, Q = w.P, w.Q
    else:
        rng = np.random.default_rng(wl.SEED_BASE + 42)
        P = w.P
        Q = w.P[np.sort(rng.choice(w.n, size=rows, replace=False))]
    res = oracle.tie_audit(P, Q, w.R)
    assert res.count == 0, res.flips[:5]
