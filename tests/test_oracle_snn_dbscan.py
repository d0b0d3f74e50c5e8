"""Pins for the plain CPU SNN (Algorithms 1-2) and the CPU DBSCAN oracle:
the Cauchy-Schwarz pruning bound Eq. (2), the two-sided sigma_2 bound Eq. (5),
the collinear best case, the Gaussian-blob efficiency model of Section 5,
exact agreement with brute force, and hand-made DBSCAN cases."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.stats import chi2, norm

import oracle
from paper_2212_07679_gb300 import workloads as wl


def _same_csr(a_offs, a_ids, a_d2, csr):
    assert np.array_equal(a_offs, csr.offsets)
    assert np.array_equal(a_ids, csr.ids)
    assert np.array_equal(a_d2.view(np.uint32), csr.dist2.view(np.uint32))


def test_cpu_snn_equals_brute_force_gmm_iso():
    work = wl.gmm_iso()
    offs, ids, d2, cand = oracle.snn_radius(work.P, work.Q, work.R)
    _same_csr(offs, ids, d2, oracle.brute_radius(work.P, work.Q, work.R))
    # pruning really prunes on this workload but keeps every neighbour
    assert cand.mean() < work.n
    assert np.all(cand >= np.diff(offs))


def test_cpu_snn_equals_brute_force_small_shapes():
    cases = [wl.gmm_aniso(n=6000, sub=2000), wl.blobs3d(n=8000, blobs=8, box=10.0)]
    for work in cases:
        offs, ids, d2, _ = oracle.snn_radius(work.P, None, work.R)
        _same_csr(offs, ids, d2, oracle.brute_radius(work.P, None, work.R))


def test_cpu_snn_exact_ties_on_a_line():
    # collinear points spaced 1 along a diagonal, R = integer spacing:
    # distances of exactly R are neighbours (inclusive boundary)
    t = np.arange(40, dtype=np.float32)
    P = np.stack([t * 3, t * 4], axis=1)       # spacing 5
    offs, ids, d2, cand = oracle.snn_radius(P, None, 5.0)
    csr = oracle.brute_radius(P, None, 5.0)
    _same_csr(offs, ids, d2, csr)
    assert csr.counts()[0] == 2 and csr.counts()[5] == 3
    # sigma_2 = 0: every candidate is a neighbour (Section 5)
    assert np.all(cand <= np.diff(offs) + 2)


def test_pruning_bound_eq2():
    rng = np.random.default_rng(11)
    P = (rng.standard_normal((800, 6)) @ rng.standard_normal((6, 6))).astype(np.float32)
    idx = oracle.snn_index(P)
    assert abs(np.linalg.norm(idx.v1) - 1.0) < 1e-12
    for i in range(0, 800, 37):
        diff = idx.X - idx.X[i]
        dist = np.sqrt(np.einsum("ij,ij->i", diff, diff))
        assert np.all(np.abs(idx.alpha - idx.alpha[i]) <= dist * (1 + 1e-12) + 1e-12)


def test_sigma2_two_sided_bound_eq5():
    rng = np.random.default_rng(12)
    P = (rng.standard_normal((600, 5)) * np.array([4, 2, 1, 0.5, 0.1])).astype(np.float32)
    idx = oracle.snn_index(P)
    s2 = idx.sigma[1]
    for i in range(0, 600, 29):
        diff = idx.X - idx.X[i]
        d2 = np.einsum("ij,ij->i", diff, diff)
        da2 = (idx.alpha - idx.alpha[i]) ** 2
        assert np.all(da2 <= d2 * (1 + 1e-10) + 1e-10)
        assert np.all(d2 <= (da2 + 2 * s2 * s2) * (1 + 1e-10) + 1e-10)


def test_principal_direction_of_elongated_blob():
    P = wl.gaussian_blob(20000, 5, 0.3, seed=13)
    idx = oracle.snn_index(P)
    assert abs(abs(idx.v1[0]) - 1.0) < 1e-3


def _blob_model(c, R, s, d):
    """P1, P2 of Section 5 by quadrature."""
    p1 = norm.cdf(c + R) - norm.cdf(c - R)
    f = lambda r: norm.pdf(r) * chi2.cdf((R * R - (r - c) ** 2) / (s * s), d - 1)
    p2, _ = integrate.quad(f, c - R, c + R)
    return p1, p2


@pytest.mark.parametrize("s,d", [(0.3, 3), (0.5, 3), (0.3, 6)])
def test_gaussian_blob_efficiency_model(s, d):
    n = 200_000
    P = wl.gaussian_blob(n, d, s, seed=14 + d)
    idx = oracle.snn_index(P)
    c, R = 0.5, 0.6
    q = np.zeros(d, np.float32)
    q[0] = c
    # query on the principal axis of the sample (the model's x_q = [c,0,..,0]
    # in principal coordinates)
    qv = (idx.mu + c * idx.v1).astype(np.float32)
    ids, _, (lo, hi), _ = oracle.snn_query(idx, qv, R)
    p1, p2 = _blob_model(c, R, s, d)
    cand = (hi - lo) / n
    ratio = len(ids) / (hi - lo)
    assert abs(cand - p1) < 0.01, (cand, p1)
    assert abs(ratio - p2 / p1) < 0.02, (ratio, p2 / p1)


def test_blob_model_monotone_in_s_and_d():
    base = _blob_model(0.5, 0.6, 0.3, 3)
    assert _blob_model(0.5, 0.6, 0.5, 3)[1] < base[1]
    assert _blob_model(0.5, 0.6, 0.3, 6)[1] < base[1]


# --------------------------------------------------------------- DBSCAN
def test_dbscan_hand_case():
    # two 4-point squares of side 1 far apart, one border point, one noise point
    P = np.array([[0, 0], [1, 0], [0, 1], [1, 1],          # cluster A (ids 0-3)
                  [10, 10], [11, 10], [10, 11], [11, 11],  # cluster B (ids 4-7)
                  [2, 0],                                  # border of A (touches id 1)
                  [50, 50]], np.float32)                   # noise
    # eps = 1: each square corner has itself + 2 neighbours = 3 -> core with minPts 3
    labels, core = oracle.dbscan(P, 1.0, 3)
    assert core.tolist() == [1, 1, 1, 1, 1, 1, 1, 1, 0, 0]
    assert labels.tolist() == [0, 0, 0, 0, 4, 4, 4, 4, 0, -1]
    l2, c2 = oracle.dbscan_bfs(P, 1.0, 3)
    assert np.array_equal(labels, l2) and np.array_equal(core, c2)


def test_dbscan_border_goes_to_smallest_core_neighbour():
    # a border point between two clusters joins the cluster of its smallest-id
    # core neighbour; a cluster's label is its smallest member id.
    # eps = 2, minPts = 4.  Cluster X = ids 0,1,2,7 near (5.5,0.25); cluster
    # Y = ids 4,5,6,8 near (0.25,0.25); id 3 at (3,0) is exactly 2 from id 0 and
    # from id 4 and has 3 neighbours counting itself, so it is a border point.
    P = np.array([[5, 0], [6, 0], [5.5, 0.5], [3, 0], [1, 0], [0, 0], [0.5, 0.5],
                  [6, 0.5], [0, 0.5]], np.float32)
    labels, core = oracle.dbscan(P, 2.0, 4)
    assert core.tolist() == [1, 1, 1, 0, 1, 1, 1, 1, 1]
    assert labels.tolist() == [0, 0, 0, 0, 4, 4, 4, 0, 4]
    l2, c2 = oracle.dbscan_bfs(P, 2.0, 4)
    assert np.array_equal(labels, l2) and np.array_equal(core, c2)


def test_dbscan_union_find_equals_bfs_random():
    for seed in range(4):
        work = wl.blobs3d(n=3000, blobs=12, box=12.0, seed=1000 + seed)
        a = oracle.dbscan(work.P, 0.4, 6)
        b = oracle.dbscan_bfs(work.P, 0.4, 6)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert (a[0] >= 0).sum() > 100 and (a[0] < 0).sum() > 10


def test_dbscan_matches_scikit_learn():
    """Pin against an independent library: scikit-learn's DBSCAN (neighbourhoods
    with dist <= eps counting the point itself, core iff at least min_samples
    of them) gives the same core points, the same noise and the same
    partition of the core points; a border point joins a cluster of one of
    its core neighbours in both (which one is the method's choice: here the
    smallest-id core neighbour's)."""
    skc = pytest.importorskip("sklearn.cluster")
    from scipy.spatial.distance import cdist
    work = wl.blobs3d(n=3000, blobs=12, box=12.0, seed=1077)
    P, eps, mp = work.P, 0.4, 6
    D = cdist(P.astype(np.float64), P.astype(np.float64))
    # no pair so close to eps that a different rounding order could flip it
    assert np.abs(D - eps).min() > 1e-9 * eps
    labels, core = oracle.dbscan(P, eps, mp)
    sk = skc.DBSCAN(eps=eps, min_samples=mp, algorithm="brute").fit(P.astype(np.float64))
    sk_core = np.zeros(len(P), dtype=bool)
    sk_core[sk.core_sample_indices_] = True
    assert np.array_equal(core.astype(bool), sk_core)
    assert np.array_equal(labels < 0, sk.labels_ < 0)
    c = core.astype(bool)
    pairs = set(zip(labels[c].tolist(), sk.labels_[c].tolist()))
    assert len(pairs) == len(set(labels[c].tolist())) == len(set(sk.labels_[c].tolist()))
    to_sk = dict(pairs)
    border = (~c) & (labels >= 0)
    for i in np.nonzero(border)[0]:
        nb_core = np.nonzero((D[i] <= eps) & c)[0]
        assert labels[i] in set(labels[nb_core].tolist())
        assert sk.labels_[i] in {to_sk[l] for l in labels[nb_core].tolist()}
    assert border.sum() > 0 and (labels < 0).sum() > 10 and len(pairs) > 5
