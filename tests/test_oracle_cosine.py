"""Pins of the cosine / angular oracle (Section 3's Euclidean reduction).

Hand cases with exactly known answers, the unit-norm and direction bounds of
the normalisation against an independent numpy norm, invariance under exact
power-of-two scaling, the closed forms of the radius mappings, and agreement
with neighbour sets computed from FP64 dot products of independently
normalised rows (away from the rounding band at the threshold)."""
import math

import numpy as np
import pytest

import oracle


def test_hand_cases():
    u = oracle.normalize_rows(np.array([[3.0, 4.0], [0.0, 0.0], [-7.0, 0.0], [0.0, 2.5e-30]], np.float32))
    assert u[0, 0] == np.float32(0.6) and u[0, 1] == np.float32(0.8)
    assert np.all(u[1] == 0.0)
    assert u[2, 0] == -1.0 and u[2, 1] == 0.0
    assert u[3, 0] == 0.0 and u[3, 1] == 1.0


def test_unit_norm_and_direction():
    rng = np.random.default_rng(11)
    for d in (1, 3, 50, 300):
        X = (rng.standard_normal((400, d)) * 10.0 ** rng.integers(-6, 7, (400, 1))).astype(np.float32)
        U = oracle.normalize_rows(X).astype(np.float64)
        norms = np.linalg.norm(U, axis=1)
        # each coordinate is one FP32 rounding of the exact unit vector
        assert np.max(np.abs(norms - 1.0)) <= 2.0 ** -24 + 1e-12
        ref = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
        assert np.all(np.abs(U - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-14)


def test_power_of_two_scaling_is_exact():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((300, 37)).astype(np.float32)
    U = oracle.normalize_rows(X)
    for k in (-20, -3, 1, 9, 20):
        assert np.array_equal(oracle.normalize_rows(X * np.float32(2.0 ** k)).view(np.uint32), U.view(np.uint32))
    assert np.array_equal(oracle.normalize_rows(-X), -U)


def test_radius_closed_forms():
    assert oracle.radius_for_cosine_similarity(1.0) == 0.0
    assert oracle.radius_for_cosine_similarity(0.0) == math.sqrt(2.0)
    assert oracle.radius_for_cosine_similarity(-1.0) == 2.0
    assert oracle.radius_for_cosine_distance(0.5) == 1.0
    assert oracle.radius_for_cosine_distance(2.0) == 2.0


def test_angles_in_the_plane():
    # unit vectors at 0, 59, 61, 120 degrees, scaled by different factors:
    # an angle bound of 60 degrees keeps 0 and 59 around the first
    ang = np.radians([0.0, 59.0, 61.0, 120.0])
    P = (np.stack([np.cos(ang), np.sin(ang)], 1) * np.array([[1.0], [3.0], [0.25], [7.0]])).astype(np.float32)
    R = oracle.radius_for_cosine_similarity(math.cos(math.radians(60.0)))
    got = oracle.cosine_radius(P, P[:1], R)
    assert list(got.row(0)[0]) == [0, 1]
    # 2 cdist at 59 degrees
    assert abs(float(got.row(0)[1][1]) - (2.0 - 2.0 * math.cos(math.radians(59.0)))) < 1e-6


def test_agrees_with_fp64_cosine_similarity():
    rng = np.random.default_rng(13)
    centres = rng.standard_normal((8, 40))
    P = (centres[rng.integers(0, 8, 900)] + 0.5 * rng.standard_normal((900, 40)))
    P = (P * rng.lognormal(0.0, 1.0, (900, 1))).astype(np.float32)
    t = 0.9
    got = oracle.cosine_radius(P, None, oracle.radius_for_cosine_similarity(t))
    Pn = P.astype(np.float64) / np.linalg.norm(P.astype(np.float64), axis=1, keepdims=True)
    cos = Pn @ Pn.T
    for i in range(0, 900, 7):
        ids, d2 = got.row(i)
        want = set(np.nonzero(cos[i] >= t)[0])
        have = set(ids.tolist())
        # outside a band of 1e-6 around the bound the two must agree
        clear = np.abs(cos[i] - t) > 1e-6
        assert {j for j in want if clear[j]} == {j for j in have if clear[j]}
        assert np.all(np.abs(d2.astype(np.float64) - (2.0 - 2.0 * cos[i, ids])) < 1e-5)
