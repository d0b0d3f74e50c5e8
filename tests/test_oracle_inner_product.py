"""Pins of the inner-product oracle: hand cases with exact dot products,
agreement with numpy's matrix product within the FP64 summation bound,
exact power-of-two scaling, sets that nest as the threshold falls, and the
augmentation identity of Section 3 that the GPU path prunes with."""
import numpy as np

import oracle


def test_hand_cases():
    P = np.array([[1, 0, 0], [0, 2, 0], [1, 1, 1], [-3, 0.5, 0], [0, 0, 0]], np.float32)
    q = np.array([[2, 1, 0]], np.float32)
    got = oracle.brute_inner_product(P, q, 1.0)
    # dot products 2, 2, 3, -5.5, 0
    assert list(got.row(0)[0]) == [0, 1, 2]
    assert list(got.row(0)[1]) == [2.0, 2.0, 3.0]
    assert oracle.brute_inner_product(P, q, 3.0).row(0)[0].tolist() == [2]
    assert oracle.brute_inner_product(P, q, 3.5).nnz == 0
    assert oracle.brute_inner_product(P, q, -10.0).nnz == 5


def test_agrees_with_matmul_within_the_summation_bound():
    rng = np.random.default_rng(21)
    for d in (1, 7, 64, 300):
        P = rng.standard_normal((500, d)).astype(np.float32)
        q = rng.standard_normal(d).astype(np.float32)
        D = oracle.dot_fp64(P, q)
        ref = P.astype(np.float64) @ q.astype(np.float64)
        A = np.abs(P.astype(np.float64)) @ np.abs(q.astype(np.float64))
        assert np.all(np.abs(D - ref) <= 2 * d * 2.0 ** -53 * A + 1e-300)


def test_power_of_two_scaling_and_nesting():
    rng = np.random.default_rng(22)
    P = rng.standard_normal((800, 20)).astype(np.float32)
    Q = rng.standard_normal((30, 20)).astype(np.float32)
    a = oracle.brute_inner_product(P, Q, 2.0)
    b = oracle.brute_inner_product(P, Q * np.float32(4.0), 8.0)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)
    assert np.array_equal(a.dist2 * np.float32(4.0), b.dist2)
    lo = oracle.brute_inner_product(P, Q, 1.0)
    for i in range(Q.shape[0]):
        assert set(a.row(i)[0].tolist()) <= set(lo.row(i)[0].tolist())


def test_augmentation_identity():
    rng = np.random.default_rng(23)
    P = rng.standard_normal((300, 12))
    q = rng.standard_normal(12)
    xi2 = np.max(np.sum(P * P, axis=1))
    Pa = np.hstack([np.sqrt(xi2 - np.sum(P * P, axis=1))[:, None], P])
    qa = np.concatenate([[0.0], q])
    lhs = np.sum((Pa - qa) ** 2, axis=1)
    rhs = xi2 + q @ q - 2 * (P @ q)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * (xi2 + q @ q)
