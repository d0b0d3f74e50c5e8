"""Pins for the FP64 brute-force oracle against facts that do not come from
the oracle itself: hand-computed cases, exact invariants, the paper's printed
return ratios (Tables 1 and 2), the closed-form distance distribution of
uniform points, and scipy's FP64 distances."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2212_07679_gb300 import workloads as wl


def _rows(csr):
    return [csr.row(i) for i in range(csr.m)]


# ---------------------------------------------------------------- hand cases
def _hand_cases(golden_dir):
    with open(os.path.join(golden_dir, "hand_cases.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("impl", ["c", "numpy"])
def test_hand_cases(golden_dir, impl):
    fn = oracle.brute_radius if impl == "c" else oracle.brute_radius_numpy
    for case in _hand_cases(golden_dir):
        P = np.asarray(case["P"], dtype=np.float32)
        Q = None if case["Q"] is None else np.asarray(case["Q"], dtype=np.float32).reshape(-1, P.shape[1])
        csr = fn(P, Q, case["R"])
        assert csr.m == len(case["ids"]), case["name"]
        for i, (ids, d2) in enumerate(_rows(csr)):
            assert ids.tolist() == case["ids"][i], (case["name"], i)
            assert d2.tolist() == [float(v) for v in case["dist2"][i]], (case["name"], i)


def test_single_pair_definition():
    # 3-4-5 in the first two coordinates of a d=3 point: S = 25 exactly
    a = np.array([3, 4, 0], np.float32)
    b = np.array([0, 0, 0], np.float32)
    assert oracle.pair_dist2(a[None], b[None], np.array([0]), np.array([0]))[0] == 25.0


# ------------------------------------------------------- exact invariants
def _random_with_ties(seed, n=300, d=5):
    rng = np.random.default_rng(seed)
    P = rng.integers(-3, 4, size=(n, d)).astype(np.float32) * 0.5   # many exact ties
    return P


def test_c_equals_numpy_bitwise():
    for seed in range(3):
        P = _random_with_ties(seed)
        Q = _random_with_ties(seed + 100, n=77)
        for R in [0.0, 1.0, 1.5, 2.0]:
            a = oracle.brute_radius(P, Q, R)
            b = oracle.brute_radius_numpy(P, Q, R)
            assert np.array_equal(a.offsets, b.offsets)
            assert np.array_equal(a.ids, b.ids)
            assert np.array_equal(a.dist2.view(np.uint32), b.dist2.view(np.uint32))


def test_self_join_symmetry_and_self_inclusion():
    rng = np.random.default_rng(5)
    P = (rng.standard_normal((500, 7)) * 3).astype(np.float32)
    csr = oracle.brute_radius(P, None, 2.5)
    pairs = {}
    for i in range(csr.m):
        ids, d2 = csr.row(i)
        assert i in ids.tolist()
        assert d2[ids.tolist().index(i)] == 0.0
        for j, s in zip(ids.tolist(), d2.tolist()):
            pairs[(i, j)] = s
    for (i, j), s in pairs.items():
        assert pairs[(j, i)] == s          # (a-b)^2 == (b-a)^2 bitwise


def test_nesting_and_infinite_radius():
    rng = np.random.default_rng(6)
    P = rng.standard_normal((400, 4)).astype(np.float32)
    Q = rng.standard_normal((50, 4)).astype(np.float32)
    prev = None
    for R in [0.3, 0.7, 1.1, 2.0]:
        csr = oracle.brute_radius(P, Q, R)
        sets = [set(csr.row(i)[0].tolist()) for i in range(csr.m)]
        if prev is not None:
            assert all(a <= b for a, b in zip(prev, sets))
        prev = sets
    big = oracle.brute_radius(P, Q, 1e30)
    assert np.all(big.counts() == P.shape[0])


def test_permutation_equivariance():
    rng = np.random.default_rng(7)
    P = rng.standard_normal((300, 6)).astype(np.float32)
    Q = rng.standard_normal((40, 6)).astype(np.float32)
    perm = rng.permutation(300)
    a = oracle.brute_radius(P, Q, 2.0)
    b = oracle.brute_radius(P[perm], Q, 2.0)
    for i in range(40):
        ia, da = a.row(i)
        ib, db = b.row(i)
        back = perm[ib]
        o = np.argsort(back)
        assert np.array_equal(back[o], ia)
        assert np.array_equal(db[o], da)


def test_translation_invariance_exact():
    # integer data shifted by a power of two: every difference is unchanged
    rng = np.random.default_rng(8)
    P = rng.integers(-20, 21, size=(200, 3)).astype(np.float32)
    a = oracle.brute_radius(P, None, 6.0)
    b = oracle.brute_radius(P + np.float32(1024.0), None, 6.0)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)
    assert np.array_equal(a.dist2, b.dist2)


def test_empty_query_set_and_single_point():
    P = np.array([[1.0, 2.0]], np.float32)
    csr = oracle.brute_radius(P, np.zeros((0, 2), np.float32), 1.0)
    assert csr.m == 0 and csr.nnz == 0
    csr = oracle.brute_radius(P, None, 0.0)
    assert csr.ids.tolist() == [0] and csr.dist2.tolist() == [0.0]


# ------------------------------------------ library routine (scipy cdist)
def test_matches_scipy_cdist_away_from_ties():
    work = wl.gmm_iso()
    S = cdist(work.Q.astype(np.float64), work.P.astype(np.float64), "sqeuclidean")
    R2 = work.R * work.R
    csr = oracle.brute_radius(work.P, work.Q, work.R)
    near = np.abs(S - R2) <= 1e-12 * R2
    for i in range(csr.m):
        got = np.zeros(work.n, bool)
        got[csr.row(i)[0]] = True
        want = S[i] <= R2
        diff = got != want
        assert not np.any(diff & ~near[i])
    # dist2 agrees with the float32 rounding of scipy's value to 1 ulp
    qi = np.repeat(np.arange(csr.m), csr.counts())
    ref = S[qi, csr.ids].astype(np.float32)
    assert np.all(np.abs(csr.dist2 - ref) <= np.spacing(ref))


# --------------------------------- printed return ratios (Tables 1 and 2)
def _ratio_excl_self(P, R):
    csr = oracle.brute_radius(P, None, R)
    n = P.shape[0]
    return 100.0 * (csr.nnz - n) / (n * n)


def _unit_square_cdf(r):
    return math.pi * r * r - 8.0 / 3.0 * r ** 3 + r ** 4 / 2.0


def _unit_cube_cdf(r):
    return 4.0 * math.pi / 3.0 * r ** 3 - 1.5 * math.pi * r ** 4 + 1.6 * r ** 5


def test_table1_d2_ratios(golden_dir):
    t = json.load(open(os.path.join(golden_dir, "table1_return_ratios.json")))["varying_n_d2"]
    n = 6000
    P = wl.uniform_cube(n, 2, seed=101)
    for Rs, printed in t["R"].items():
        R = float(Rs)
        got = _ratio_excl_self(P, R)
        closed = 100.0 * _unit_square_cdf(R)
        ref = float(np.mean(printed))
        # pair count ~ n^2 p / 2: relative sampling sd <= 1.5% here; 6% slack
        assert abs(got - ref) <= 0.06 * ref, (R, got, ref)
        assert abs(got - closed) <= 0.06 * closed, (R, got, closed)
        assert abs(ref - closed) <= 0.02 * closed      # the paper agrees with the closed form


def test_table1_d50_ratios(golden_dir):
    t = json.load(open(os.path.join(golden_dir, "table1_return_ratios.json")))["varying_n_d50"]
    n = 8000
    P = wl.uniform_cube(n, 50, seed=102)
    for Rs, printed in t["R"].items():
        R = float(Rs)
        got = _ratio_excl_self(P, R)
        ref = float(np.mean(printed))
        pairs = ref / 100.0 * n * n / 2
        tol = 6.0 / math.sqrt(pairs) + 0.03
        assert abs(got - ref) <= tol * ref, (R, got, ref)


def test_table1_varying_d(golden_dir):
    t = json.load(open(os.path.join(golden_dir, "table1_return_ratios.json")))["varying_d_n10000"]
    n = 3000
    for di, d in enumerate(t["d"][:3]):
        P = wl.uniform_cube(n, d, seed=103 + d)
        for Rs, printed in t["R"].items():
            ref = printed[di]
            got = _ratio_excl_self(P, float(Rs))
            if ref == 0:
                assert got <= 1e-3
            elif ref >= 99.99:
                assert got >= 99.9
            elif ref > 0.1:
                assert abs(got - ref) <= 0.08 * ref + 0.05, (d, Rs, got, ref)


def test_table2_d3_ratios(golden_dir):
    t = json.load(open(os.path.join(golden_dir, "table2_return_ratios.json")))
    P = wl.uniform_cube(6000, 3, seed=104)
    for Rs, printed in t["varying_n_d3"]["R"].items():
        R = float(Rs)
        got = _ratio_excl_self(P, R)
        ref = float(np.mean(printed))
        closed = 100.0 * _unit_cube_cdf(R)
        assert abs(got - closed) <= 0.08 * closed, (R, got, closed)
        assert abs(ref - closed) <= 0.1 * closed
    for di, d in enumerate(t["varying_d_n10000"]["d"]):
        P = wl.uniform_cube(5000, d, seed=105 + d)
        for Rs, printed in t["varying_d_n10000"]["R"].items():
            ref = printed[di]
            if ref < 0.04:
                continue
            got = _ratio_excl_self(P, float(Rs))
            assert abs(got - ref) <= 0.12 * ref, (d, Rs, got, ref)


def test_radius_rows_equals_brute_force():
    """The row-sampled oracle (a float64 product discards pairs certainly
    outside, the FP64 definition decides the rest) returns exactly the rows
    of the full brute force: random clusters, exact ties on an integer grid
    (S == R^2 on the boundary), duplicates, negative and large coordinates,
    and out-of-sample queries."""
    rng = np.random.default_rng(91)
    cases = []
    P = (rng.standard_normal((3000, 20)) + 50.0 * rng.standard_normal((5, 20))[rng.integers(0, 5, 3000)])
    cases.append((P.astype(np.float32), None, 4.5))
    g = np.stack(np.meshgrid(np.arange(12), np.arange(12), np.arange(12)), -1).reshape(-1, 3) - 6
    cases.append((g.astype(np.float32), None, 2.0))
    dup = np.repeat(rng.standard_normal((40, 7)), 9, axis=0).astype(np.float32)
    cases.append((dup, None, 0.0))
    P2 = (rng.standard_normal((2000, 64)) * 1e3).astype(np.float32)
    Q2 = (rng.standard_normal((300, 64)) * 1e3).astype(np.float32)
    cases.append((P2, Q2, float(np.sqrt(2 * 64) * 1e3 * 0.9)))
    for P, Q, R in cases:
        m = P.shape[0] if Q is None else Q.shape[0]
        rows = rng.choice(m, size=min(m, 257), replace=False)
        got = oracle.radius_rows(P, Q, rows, R)
        ref = oracle.brute_radius(P, (P if Q is None else Q)[rows], R)
        assert np.array_equal(got.offsets, ref.offsets)
        assert np.array_equal(got.ids, ref.ids)
        assert np.array_equal(got.dist2.view(np.uint32), ref.dist2.view(np.uint32))
    with pytest.raises(ValueError):
        oracle.radius_rows(P2, None, [0], 1.0, margin=1e-16)


def test_radius_grid_equals_brute_force():
    """The grid-cell evaluation of the definition returns exactly the full
    brute force in d = 1..4: clusters, exact ties on an integer grid at R = 1
    and R = 2, duplicates at R = 0, negative and offset coordinates, and
    out-of-sample queries."""
    rng = np.random.default_rng(92)
    cases = []
    for d in (1, 2, 3, 4):
        P = (rng.standard_normal((2500, d)) + 8.0 * rng.standard_normal((4, d))[rng.integers(0, 4, 2500)])
        cases.append((P.astype(np.float32), None, 0.35))
        Q = (rng.standard_normal((400, d)) * 6.0 - 100.0 * (d == 2)).astype(np.float32)
        cases.append(((P - 100.0 * (d == 2)).astype(np.float32), Q, 0.8))
    g = np.stack(np.meshgrid(np.arange(10), np.arange(10), np.arange(10)), -1).reshape(-1, 3) - 5
    cases.append((g.astype(np.float32), None, 1.0))
    cases.append((g.astype(np.float32), None, 2.0))
    dup = np.repeat(rng.standard_normal((50, 3)), 6, axis=0).astype(np.float32)
    cases.append((dup, None, 0.0))
    for P, Q, R in cases:
        got = oracle.radius_grid(P, Q, R, chunk=777)
        ref = oracle.brute_radius(P, Q, R)
        assert np.array_equal(got.offsets, ref.offsets)
        assert np.array_equal(got.ids, ref.ids)
        assert np.array_equal(got.dist2.view(np.uint32), ref.dist2.view(np.uint32))
    with pytest.raises(ValueError):
        oracle.radius_grid(np.zeros((3, 5), np.float32), None, 1.0)
