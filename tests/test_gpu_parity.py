"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Neighbour sets, their order and the squared distances must match the oracle
bit for bit (ids ascending per row; dist2 = (float)S with S the FP64
direct-difference sum).  Small cases span several 128-row tiles and a ragged
tail; the full-size self-join of the 1e6-point mixture is checked on sampled
rows and by properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_2212_07679_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16"]


@pytest.fixture(scope="module")
def snn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_07679_gb300 import snn as mod
    return mod


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def assert_csr_equal(got, ref, what=""):
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    assert off.shape == ref.offsets.shape, what
    if not np.array_equal(off, ref.offsets):
        bad = np.nonzero(np.diff(off) != np.diff(ref.offsets))[0]
        raise AssertionError(f"{what}: row counts differ at rows {bad[:10]} "
                             f"(got {np.diff(off)[bad[:5]]}, want {np.diff(ref.offsets)[bad[:5]]})")
    assert np.array_equal(idx, ref.ids), what
    assert np.array_equal(d2.view(np.uint32), ref.dist2.view(np.uint32)), what


def _run(snn, P, Q, R, prec):
    ix = snn.Index(_dev(P))
    try:
        return ix.query(None if Q is None else _dev(Q), R, precision=prec, stats=True)
    except snn.SNNError as e:
        if e.status == snn.SNN_ENOTSUP:
            pytest.skip(f"{prec} not available: {e}")
        raise


# ------------------------------------------------------------- hand cases
@pytest.mark.parametrize("prec", PRECS)
def test_hand_cases(snn, golden_dir, prec):
    import json
    import os
    cases = json.load(open(os.path.join(golden_dir, "hand_cases.json")))["cases"]
    for case in cases:
        P = np.asarray(case["P"], dtype=np.float32)
        Q = None if case["Q"] is None else np.asarray(case["Q"], np.float32).reshape(-1, P.shape[1])
        got = _run(snn, P, Q, case["R"], prec)
        assert_csr_equal(got, oracle.brute_radius(P, Q, case["R"]), case["name"])


# -------------------------------------------------- workloads, small sizes
@pytest.mark.parametrize("prec", PRECS)
def test_gmm_iso_full_size(snn, prec):
    w = wl.gmm_iso()
    got = _run(snn, w.P, w.Q, w.R, prec)
    assert_csr_equal(got, oracle.brute_radius(w.P, w.Q, w.R), "gmm_iso")
    st = got.stats
    assert st["band_pairs"] >= st["candidates"] >= st["nnz"] == got.nnz
    assert st["survivors"] >= st["nnz"]


@pytest.mark.parametrize("prec", PRECS)
def test_stats_without_candidate_count(snn, prec):
    """stats="phases" (SNN_STATS_NO_CANDIDATES) skips the candidate-range
    count only: the same CSR and counters, candidates = -1."""
    w = wl.gmm_iso()
    X = _dev(w.P)
    Q = _dev(w.Q)
    full = snn.Index(X).query(Q, w.R, precision=prec, stats=True)
    light = snn.Index(X).query(Q, w.R, precision=prec, stats="phases")
    assert light.stats["candidates"] == -1 and full.stats["candidates"] > 0
    for k in ("band_pairs", "survivors", "nnz", "exact_fp64", "split_used", "precision_used"):
        assert light.stats[k] == full.stats[k], k
    assert torch.equal(light.offsets, full.offsets) and torch.equal(light.indices, full.indices)
    assert torch.equal(light.dist2.view(torch.int32), full.dist2.view(torch.int32))
    with pytest.raises(ValueError):
        snn.Index(X).query(Q, w.R, precision=prec, stats="all")


@pytest.mark.parametrize("prec", PRECS)
def test_gmm_aniso_self_join_small(snn, prec):
    w = wl.gmm_aniso(n=20011, sub=3000)
    got = _run(snn, w.P, None, w.R, prec)
    assert_csr_equal(got, oracle.brute_radius(w.P, None, w.R), "gmm_aniso")


@pytest.mark.parametrize("prec", PRECS)
def test_blobs3d_self_join_small(snn, prec):
    w = wl.blobs3d(n=20000, blobs=16, box=20.0)
    got = _run(snn, w.P, None, w.R, prec)
    assert_csr_equal(got, oracle.brute_radius(w.P, None, w.R), "blobs3d")


@pytest.mark.parametrize("prec", PRECS)
def test_lowrank_img_self_join_small(snn, prec):
    w = wl.lowrank_img(n=3001, sub=1500)
    got = _run(snn, w.P, None, w.R, prec)
    assert_csr_equal(got, oracle.brute_radius(w.P, None, w.R), "lowrank_img")


@pytest.mark.parametrize("prec", PRECS)
def test_out_of_sample_queries(snn, prec):
    rng = np.random.default_rng(21)
    P = (rng.standard_normal((7000, 12)) * 2).astype(np.float32)
    Q = (rng.standard_normal((1500, 12)) * 2.5 + 0.3).astype(np.float32)
    for R in [0.0, 1.5, 3.0]:
        got = _run(snn, P, Q, R, prec)
        assert_csr_equal(got, oracle.brute_radius(P, Q, R), f"oos R={R}")


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(snn, prec):
    rng = np.random.default_rng(22)
    cases = []
    cases.append(("n=1", np.array([[1.0, 2.0, 3.0]], np.float32), None, 0.0))
    cases.append(("d=1", rng.standard_normal((700, 1)).astype(np.float32), None, 0.01))
    line = np.arange(300, dtype=np.float32)[:, None] * np.array([[3, 4]], np.float32)
    cases.append(("line exact ties", line, None, 5.0))
    dup = np.repeat(rng.standard_normal((20, 6)).astype(np.float32), 15, axis=0)
    cases.append(("duplicates R=0", dup, None, 0.0))
    cases.append(("d=17 ragged", rng.integers(-2, 3, (777, 17)).astype(np.float32), None, 2.0))
    off = (rng.standard_normal((900, 5)) + 1e4).astype(np.float32)
    cases.append(("large offset", off, None, 1.2))
    # squared distances in the FP32 subnormal range (the compensated tier
    # underflows there and must hand the pair to the FP64 loop)
    tiny = np.array([[0, 0], [2.0 ** -74, 0], [0, 2.0 ** -60], [1e-30, 1e-30], [2.0 ** -80, 2.0 ** -80]],
                    np.float32)
    cases.append(("subnormal distances", tiny, None, 1e-20))
    grid = np.stack(np.meshgrid(np.arange(12), np.arange(12), np.arange(12)), -1).reshape(-1, 3)
    cases.append(("integer grid exact ties", grid.astype(np.float32), None, 1.0))
    cases.append(("all within R (long rows)", rng.random((4500, 3)).astype(np.float32), None, 2.0))
    Q = rng.standard_normal((0, 4)).astype(np.float32)
    cases.append(("m=0", rng.standard_normal((50, 4)).astype(np.float32), Q, 1.0))
    for name, P, Qc, R in cases:
        got = _run(snn, P, Qc, R, prec)
        assert_csr_equal(got, oracle.brute_radius(P, Qc, R), name)


def test_index_arrays(snn):
    w = wl.gmm_aniso(n=30000, sub=2000)
    ix = snn.Index(_dev(w.P))
    v = ix.view()
    alpha = v["alpha"].cpu().numpy()
    order = v["order"].cpu().numpy()
    assert np.all(np.diff(alpha) >= 0)
    assert np.array_equal(np.sort(order), np.arange(w.n))
    assert np.array_equal(v["points"].cpu().numpy(), w.P[order])
    v1 = v["v1"].cpu().numpy()
    assert abs(np.linalg.norm(v1) - 1.0) < 1e-12
    ref = oracle.snn_index(w.P)
    assert abs(abs(float(v1 @ ref.v1)) - 1.0) < 1e-3
    assert np.allclose(v["mu"].cpu().numpy(), ref.mu, rtol=0, atol=1e-9)
    # the centre is the FP32 rounding of the mean; scores are within the
    # recorded bound of the FP64 projection of the points shifted by it
    c = v["centre"].cpu().numpy()
    assert np.array_equal(c, v["mu"].cpu().numpy().astype(np.float32))
    a64 = (w.P[order].astype(np.float64) - c.astype(np.float64)) @ v1
    assert np.max(np.abs(alpha - a64)) <= v["alpha_err"]


@pytest.mark.parametrize("d,n", [(100, 3000), (784, 5000), (130, 257)])
def test_index_arrays_tensor_core_gram(snn, d, n):
    """d > 64: the Gram matrix and the squarings run on the tensor cores.  The
    first direction must agree with the oracle's (SVD of the centred data) and
    the scores must stay within their recorded bound."""
    if d == 784:
        w = wl.lowrank_img(n=n, sub=1500)
        P = w.P
    else:
        rng = np.random.default_rng(d)
        # a dominant direction with a clear gap to the second
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        P = (rng.standard_normal((n, d)) + 6.0 * rng.standard_normal((n, 1)) * u + 3.0).astype(np.float32)
    ix = snn.Index(_dev(P))
    v = ix.view()
    order = v["order"].cpu().numpy()
    alpha = v["alpha"].cpu().numpy()
    assert np.all(np.diff(alpha) >= 0)
    assert np.array_equal(np.sort(order), np.arange(n))
    v1 = v["v1"].cpu().numpy()
    assert abs(np.linalg.norm(v1) - 1.0) < 1e-12
    ref = oracle.snn_index(P)
    assert abs(abs(float(v1 @ ref.v1)) - 1.0) < 1e-3
    c = v["centre"].cpu().numpy().astype(np.float64)
    a64 = (P[order].astype(np.float64) - c) @ v1
    assert np.max(np.abs(alpha - a64)) <= v["alpha_err"]


@pytest.mark.parametrize("prec", PRECS)
def test_high_d_degenerate_and_offset(snn, prec):
    """d > 64 special cases of the tensor-core Gram: all points equal (C = 0,
    v1 = e1), a large common offset, and a row count that is not a multiple
    of the 64-row k-block."""
    rng = np.random.default_rng(31)
    same = np.repeat(rng.standard_normal((1, 96)).astype(np.float32), 333, axis=0)
    got = _run(snn, same, None, 0.0, prec)
    assert_csr_equal(got, oracle.brute_radius(same, None, 0.0), "identical d=96")
    v1 = snn.Index(_dev(same)).view()["v1"].cpu().numpy()
    assert v1[0] == 1.0 and np.all(v1[1:] == 0.0)
    off = (rng.standard_normal((1111, 80)) * 0.5 + 3e3).astype(np.float32)
    got = _run(snn, off, None, 3.0, prec)
    assert_csr_equal(got, oracle.brute_radius(off, None, 3.0), "offset d=80")


@pytest.mark.parametrize("prec", PRECS)
def test_long_rows_exact_ties(snn, prec):
    """Binary vectors: squared distances are integers, so many pairs sit
    exactly on R^2 and take the FP64 fallback of the lane-group decision
    (8 lanes per survivor at d = 72, 32 lanes at d = 200)."""
    rng = np.random.default_rng(41)
    for d, n, R in [(72, 600, 6.0), (200, 500, 10.0)]:
        P = rng.integers(0, 2, (n, d)).astype(np.float32)
        got = _run(snn, P, None, R, prec)
        assert_csr_equal(got, oracle.brute_radius(P, None, R), f"binary d={d}")
        assert got.stats["exact_fp64"] > 0


def test_invalid_inputs(snn):
    P = np.random.default_rng(23).standard_normal((100, 4)).astype(np.float32)
    P[17, 2] = np.nan
    with pytest.raises(snn.SNNError) as e:
        snn.Index(_dev(P))
    assert e.value.status == snn.SNN_EINVAL
    ix = snn.Index(_dev(np.nan_to_num(P)))
    with pytest.raises(snn.SNNError):
        ix.query(None, -1.0)
    with pytest.raises(snn.SNNError):
        ix.query(None, float("inf"))
    Q = np.ones((5, 4), np.float32)
    Q[3, 1] = np.inf
    with pytest.raises(snn.SNNError) as e:
        ix.query(_dev(Q), 1.0)
    assert e.value.status == snn.SNN_EINVAL


def test_deterministic_repeat(snn):
    w = wl.gmm_aniso(n=15000, sub=2000)
    a = _run(snn, w.P, None, w.R, "fp32")
    b = _run(snn, w.P, None, w.R, "fp32")
    assert torch.equal(a.offsets, b.offsets) and torch.equal(a.indices, b.indices)
    assert torch.equal(a.dist2, b.dist2)


# ------------------------------------------------------------- DBSCAN
def test_dbscan_small(snn):
    w = wl.blobs3d(n=30000, blobs=20, box=25.0)
    labels, core = snn.dbscan(_dev(w.P), 0.4, 10)
    ref_l, ref_c = oracle.dbscan(w.P, 0.4, 10)
    assert np.array_equal(core.cpu().numpy(), ref_c)
    assert np.array_equal(labels.cpu().numpy(), ref_l)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dbscan_border_points_between_clusters(snn, prec):
    """Border points reachable from two clusters join the cluster of their
    smallest-id core neighbour (the GPU scans unsorted neighbourhoods in
    sorted positions); the hand case of two clusters sharing a border point,
    under row permutations that reorder the ids against the projections, and
    chains of points alternating between two clusters."""
    base = np.array([[5, 0], [6, 0], [5.5, 0.5], [3, 0], [1, 0], [0, 0], [0.5, 0.5],
                     [6, 0.5], [0, 0.5]], np.float32)
    rng = np.random.default_rng(61)
    for perm in [np.arange(len(base))] + [rng.permutation(len(base)) for _ in range(4)]:
        P = np.ascontiguousarray(base[perm])
        labels, core = snn.dbscan(_dev(P), 2.0, 4, precision=prec)
        ref_l, ref_c = oracle.dbscan(P, 2.0, 4)
        assert np.array_equal(core.cpu().numpy(), ref_c), perm
        assert np.array_equal(labels.cpu().numpy(), ref_l), perm
    # many border points: pairs of dense 1-D clusters with sparse bridges
    pts = []
    for k in range(40):
        x0 = 10.0 * k
        pts.append(np.stack([x0 + rng.uniform(0, 1.0, 30), rng.uniform(0, 0.3, 30)], 1))
        pts.append(np.stack([x0 + 2.6 + rng.uniform(0, 1.0, 30), rng.uniform(0, 0.3, 30)], 1))
        pts.append(np.stack([x0 + 1.8 + rng.uniform(-0.05, 0.05, 3), rng.uniform(0, 0.3, 3)], 1))
    P = np.concatenate(pts).astype(np.float32)
    P = P[rng.permutation(len(P))]
    labels, core = snn.dbscan(_dev(P), 0.9, 8, precision=prec)
    ref_l, ref_c = oracle.dbscan(P, 0.9, 8)
    assert np.array_equal(core.cpu().numpy(), ref_c)
    assert np.array_equal(labels.cpu().numpy(), ref_l)
    assert (ref_c == 0).sum() > 0 and len(np.unique(ref_l[ref_l >= 0])) > 40


# ------------------------------------------------------------ batches
def test_batch_matches_oracle(snn):
    # one call, one persistent scoring launch for all sets: ragged n and d
    # (2, 3, 8, 32), out-of-sample queries, per-set radius
    sets = wl.ragged_batch(sets=12, n_lo=500, n_hi=6000, seed=99)
    idx = [snn.Index(_dev(s.P)) for s in sets]
    before = snn.launch_count()
    outs = snn.query_batch(idx, [_dev(s.Q) for s in sets], [s.R for s in sets])
    launches = snn.launch_count() - before
    assert launches < 60          # independent of the number of sets
    for s, got in zip(sets, outs):
        assert_csr_equal(got, oracle.brute_radius(s.P, s.Q, s.R), s.name)


def test_batch_mixed_sets(snn):
    rng = np.random.default_rng(98)
    cases = []
    for k, (n, d) in enumerate([(3000, 2), (2500, 17), (4000, 8), (1200, 40), (900, 3), (50, 5)]):
        P = (rng.standard_normal((n, d)) * (1 + k)).astype(np.float32)
        if k % 2 == 0:
            cases.append((P, None, 0.9 + 0.2 * k))                      # self-join
        else:
            Q = (rng.standard_normal((n // 3, d)) * (1 + k)).astype(np.float32)
            cases.append((P, Q, 1.1 + 0.1 * k))
    cases.append((rng.standard_normal((700, 4)).astype(np.float32),
                  np.zeros((0, 4), np.float32), 1.0))                   # no queries
    dup = np.repeat(rng.standard_normal((30, 6)).astype(np.float32), 7, axis=0)
    cases.append((dup, None, 0.0))                                       # R = 0, duplicates
    idx = [snn.Index(_dev(P)) for P, _, _ in cases]
    Qs = [None if Q is None else _dev(Q) for _, Q, _ in cases]
    outs = snn.query_batch(idx, Qs, [R for _, _, R in cases])
    for k, ((P, Q, R), got) in enumerate(zip(cases, outs)):
        assert_csr_equal(got, oracle.brute_radius(P, Q, R), f"set {k}")
    # the per-set results are slices of one allocation: free them out of order
    for k in [3, 0, 7, 1, 6, 2, 5, 4]:
        outs[k] = None
    del outs


# ------------------------------------------------- full size (sampled)
@pytest.mark.slow
def test_full_size_self_join_sampled(snn):
    w = wl.gmm_aniso()
    ix = snn.Index(_dev(w.P))
    got = ix.query(None, w.R, stats=True)
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    rng = np.random.default_rng(24)
    rows = rng.choice(w.n, size=64, replace=False)
    ref = oracle.brute_radius(w.P, w.P[rows], w.R)
    for t, r in enumerate(rows):
        ri, rd = ref.row(t)
        a, b = off[r], off[r + 1]
        assert np.array_equal(idx[a:b], ri)
        assert np.array_equal(d2[a:b].view(np.uint32), rd.view(np.uint32))
    # properties at full size: self-inclusion with dist2 0, ascending rows,
    # symmetry of the self-join
    counts = np.diff(off)
    rowid = np.repeat(np.arange(w.n), counts)
    assert np.all(counts >= 1)
    assert np.all((idx[1:] > idx[:-1]) | (rowid[1:] != rowid[:-1]))
    self_hits = idx == rowid
    assert self_hits.sum() == w.n and np.all(d2[self_hits] == 0)
    fwd = rowid.astype(np.int64) * w.n + idx
    bwd = idx.astype(np.int64) * w.n + rowid
    assert np.array_equal(np.sort(fwd), np.sort(bwd))


def test_exact_ties_take_the_fp64_path(snn):
    # integer grid with R = 2: many pairs sit exactly on the boundary S == R^2,
    # which the compensated FP32 tier cannot settle; they must be decided by
    # the FP64 loop and included (inclusive radius)
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), np.arange(9)), -1).reshape(-1, 3)
    P = g.astype(np.float32) * np.float32(0.5)
    got = _run(snn, P, None, 1.0, "fp32")
    assert_csr_equal(got, oracle.brute_radius(P, None, 1.0), "half-integer grid")
    assert got.stats["exact_fp64"] > 0
    # random data: the FP64 loop is (almost) never needed
    w = wl.gmm_aniso(n=20000, sub=2000)
    got = _run(snn, w.P, None, w.R, "fp32")
    assert got.stats["exact_fp64"] <= max(2, got.stats["survivors"] // 10000)


def test_launch_counter_moves(snn):
    before = snn.launch_count()
    _run(snn, np.random.default_rng(1).standard_normal((500, 3)).astype(np.float32), None, 0.5, "fp32")
    assert snn.launch_count() > before


@pytest.mark.parametrize("d", [5, 23, 40, 55, 100, 300])
@pytest.mark.parametrize("spread", [1.0, 30.0])
def test_tensor_core_shapes(snn, d, spread):
    # covers every tensor-core kernel shape: one 32- or 64-column k-block with
    # the query tile resident (d + 9 <= 64) or streamed 64-column k-blocks,
    # and both the two- and three-part BF16 splits (cluster spread relative to
    # R decides the split)
    rng = np.random.default_rng(100 + d)
    centres = rng.uniform(-spread, spread, size=(6, d))
    lab = rng.integers(0, 6, size=5000)
    P = (centres[lab] + rng.standard_normal((5000, d))).astype(np.float32)
    Q = (centres[rng.integers(0, 6, size=700)] + rng.standard_normal((700, d))).astype(np.float32)
    R = float(np.sqrt(2.0 * d) * 0.8)
    for q in (None, Q):
        got = _run(snn, P, q, R, "bf16")
        assert_csr_equal(got, oracle.brute_radius(P, q, R), f"d={d} spread={spread}")


def _check_sampled_rows(got, P, Q, R, rows):
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    Qs = P[rows] if Q is None else Q[rows]
    ref = oracle.brute_radius(P, Qs, R)
    for t, r in enumerate(rows):
        ri, rd = ref.row(t)
        a, b = off[r], off[r + 1]
        assert np.array_equal(idx[a:b], ri), r
        assert np.array_equal(d2[a:b].view(np.uint32), rd.view(np.uint32)), r


@pytest.mark.slow
def test_full_size_self_join_sampled_bf16(snn):
    w = wl.gmm_aniso()
    got = snn.Index(_dev(w.P)).query(None, w.R, precision="bf16")
    rows = np.random.default_rng(25).choice(w.n, size=48, replace=False)
    _check_sampled_rows(got, w.P, None, w.R, rows)
    assert got.nnz == int(got.offsets[-1])


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECS)
def test_full_size_lowrank_img_sampled(snn, prec):
    w = wl.lowrank_img()
    got = snn.Index(_dev(w.P)).query(None, w.R, precision=prec, stats=True)
    rows = np.random.default_rng(26).choice(w.n, size=24, replace=False)
    _check_sampled_rows(got, w.P, None, w.R, rows)
    # symmetry of the whole self-join
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy().astype(np.int64)
    rowid = np.repeat(np.arange(w.n, dtype=np.int64), np.diff(off))
    assert np.array_equal(np.sort(rowid * w.n + idx), np.sort(idx * w.n + rowid))


@pytest.mark.slow
def test_full_size_lowrank_img_whole_csr(snn):
    """The 70,000 x 784 self-join at full size, every row: the rows' entries
    at columns from their 4,096-row block onwards are compared with the
    oracle's (oracle.radius_rows against the points from that block on), and
    the whole CSR is symmetric, so every pair is checked once.  The default
    16-bit scorer here keeps one FP16 part per row; the pairs nearest to R^2
    that the oracle returns show the check reaches the boundary."""
    w = wl.lowrank_img()
    got = snn.Index(_dev(w.P)).query(None, w.R, precision="bf16", stats=True)
    assert got.stats["split_used"] == snn.SNN_SPLIT_FP16X1
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    n, R2 = w.n, float(np.float64(w.R) * np.float64(w.R))
    step, checked, near = 4096, 0, 0
    for a in range(0, n, step):
        b = min(n, a + step)
        ref = oracle.radius_rows(w.P[a:], w.P, np.arange(a, b), w.R)
        for t, r in enumerate(range(a, b)):
            ri, rd = ref.row(t)
            lo, hi = off[r], off[r + 1]
            sel = idx[lo:hi] >= a
            assert np.array_equal(idx[lo:hi][sel], ri + a), r
            assert np.array_equal(d2[lo:hi][sel].view(np.uint32), rd.view(np.uint32)), r
            checked += len(ri)
            near += int(np.count_nonzero(rd.astype(np.float64) >= R2 * (1.0 - 1e-6)))
    rowid = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    ii = idx.astype(np.int64)
    assert np.array_equal(np.sort(rowid * n + ii), np.sort(ii * n + rowid))
    # every pair is compared at least once (pairs inside one block twice)
    assert (got.nnz + n) // 2 <= checked <= got.nnz
    assert near > 0


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECS)
def test_full_size_dbscan_labels(snn, prec):
    """DBSCAN on the 500,000-point particle set (eps 0.4, minPts 10) at full
    size: labels and core flags equal the oracle's DBSCAN element by element,
    and the self-join under it equals the oracle's neighbour lists (every
    pair in adjacent grid cells evaluated by the FP64 definition)."""
    w = wl.blobs3d()
    eps, min_pts = w.R, w.extra["min_pts"]
    ref_csr = oracle.radius_grid(w.P, None, eps)
    ref_lab, ref_core = oracle.dbscan(w.P, eps, min_pts, csr=ref_csr)
    X = _dev(w.P)
    labels, core = snn.dbscan(X, eps, min_pts, precision=prec)
    lab = labels.cpu().numpy()
    cr = core.cpu().numpy()
    assert np.array_equal(cr, ref_core)
    bad = np.nonzero(lab != ref_lab)[0]
    assert bad.size == 0, f"{bad.size} labels differ, first at {bad[:5]}"
    got = snn.Index(X).query(None, eps, precision=prec)
    assert_csr_equal(got, ref_csr, f"blobs3d self-join {prec}")


@pytest.mark.slow
def test_full_size_dbscan_sampled(snn):
    w = wl.blobs3d()
    eps, min_pts = w.R, w.extra["min_pts"]
    labels, core = snn.dbscan(_dev(w.P), eps, min_pts)
    labels = labels.cpu().numpy()
    core = core.cpu().numpy().astype(bool)
    n = w.n
    # canonical labels: a cluster's label is one of its members, its smallest
    lab = labels[labels >= 0]
    assert np.all(labels[np.unique(lab)] == np.unique(lab))
    assert np.all((labels < 0) | (labels <= np.arange(n)))
    assert np.all(labels[core] >= 0)
    rows = np.random.default_rng(27).choice(n, size=300, replace=False)
    ref = oracle.brute_radius(w.P, w.P[rows], eps)
    for t, r in enumerate(rows):
        nb = ref.row(t)[0]
        assert core[r] == (len(nb) >= min_pts), r
        core_nb = nb[core[nb]]
        if core[r]:
            # every core neighbour is in the same cluster
            assert np.all(labels[core_nb] == labels[r]), r
        elif len(core_nb):
            assert labels[r] == labels[core_nb.min()], r
        else:
            assert labels[r] == -1, r


@pytest.mark.slow
def test_full_size_ragged_batch_sampled(snn):
    sets = wl.ragged_batch()
    idx = [snn.Index(_dev(s.P)) for s in sets]
    outs = snn.query_batch(idx, [_dev(s.Q) for s in sets], [s.R for s in sets])
    rng = np.random.default_rng(28)
    for s, got in zip(sets, outs):
        rows = rng.choice(s.m, size=min(2, s.m), replace=False)
        _check_sampled_rows(got, s.P, s.Q, s.R, rows)
        assert got.m == s.m


def test_to_host_pinned_copies(snn):
    """CSR.to_host copies into pinned, reused host buffers; the copies equal
    the device arrays, and a larger result regrows the buffers."""
    rng = np.random.default_rng(71)
    P = rng.standard_normal((3000, 5)).astype(np.float32)
    ix = snn.Index(_dev(P))
    bufs = snn.HostBuffers()
    for R in (0.5, 1.2, 0.8):
        out = ix.query(None, R, precision="bf16")
        host = out.to_host(bufs)
        assert host.offsets.is_pinned() and host.indices.is_pinned() and host.dist2.is_pinned()
        assert host.nnz == out.nnz and host.m == out.m
        assert np.array_equal(host.offsets.numpy(), out.offsets.cpu().numpy())
        assert np.array_equal(host.indices.numpy(), out.indices.cpu().numpy())
        assert np.array_equal(host.dist2.numpy().view(np.uint32), out.dist2.cpu().numpy().view(np.uint32))
        assert_csr_equal(out, oracle.brute_radius(P, None, R), f"R={R}")


@pytest.mark.parametrize("keys64", ["0", "1"])
def test_row_sort_key_widths(snn, monkeypatch, keys64):
    """Rows of every length class (warp sorts up to 512, block sort up to
    4,096, radix beyond) with the 32-bit sort keys (id, position) and with
    the 64-bit packed keys forced by SNN_SORT_KEYS64: both equal the oracle."""
    monkeypatch.setenv("SNN_SORT_KEYS64", keys64)
    rng = np.random.default_rng(43)
    parts = [rng.normal(0.0, 0.01, (5000, 3)),                 # rows of ~5,000 (radix)
             rng.normal(5.0, 0.01, (1500, 3)),                 # ~1,500 (block sort)
             rng.normal(-5.0, 0.3, (3000, 3)),                 # tens to hundreds (warp sorts)
             rng.uniform(-20.0, 20.0, (2000, 3))]              # short rows
    P = np.concatenate(parts).astype(np.float32)
    P = P[rng.permutation(len(P))]
    got = _run(snn, P, None, 0.2, "bf16")
    ref = oracle.brute_radius(P, None, 0.2)
    lens = np.diff(ref.offsets)
    assert lens.max() > 4096 and ((lens > 512) & (lens <= 4096)).any() and (lens <= 32).any()
    assert_csr_equal(got, ref, f"keys64={keys64}")


@pytest.mark.parametrize("keys64", ["0", "1"])
@pytest.mark.parametrize("prec", PRECS)
def test_row_lengths_at_sort_class_edges(snn, monkeypatch, keys64, prec):
    """Rows whose lengths sit on both sides of every per-row sort class edge
    (8, 16, 32, 64, 128, 256, 512): well separated tight clusters of k points
    give k rows of exactly k entries; self-join and out-of-sample queries."""
    monkeypatch.setenv("SNN_SORT_KEYS64", keys64)
    rng = np.random.default_rng(47)
    sizes = [1, 2, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257,
             511, 512, 513]
    centres = rng.permutation(len(sizes))[:, None] * np.array([[100.0, -50.0, 25.0]])
    P = np.concatenate([c + rng.normal(0.0, 0.01, (k, 3)) for c, k in zip(centres, sizes)])
    P = P[rng.permutation(len(P))].astype(np.float32)
    got = _run(snn, P, None, 1.0, prec)
    ref = oracle.brute_radius(P, None, 1.0)
    assert sorted(set(np.diff(ref.offsets).tolist())) == sorted(sizes)
    assert_csr_equal(got, ref, f"self-join keys64={keys64}")
    Q = P[rng.permutation(len(P))[:700]] + np.float32(0.001)
    got = _run(snn, P, Q, 1.0, prec)
    assert_csr_equal(got, oracle.brute_radius(P, Q, 1.0), f"queries keys64={keys64}")


@pytest.mark.parametrize("split", ["bf16x2", "bf16x3", "fp16x2", "fp16x1"])
@pytest.mark.parametrize("d,spread", [(12, 40.0), (16, 3.0), (40, 10.0), (100, 2.0), (300, 6.0)])
def test_tensor_core_shapes_forced_split(snn, monkeypatch, split, d, spread):
    """Every 16-bit operand split (SNN_TC_SPLIT) on every kernel shape,
    whatever the automatic choice would be (one FP16 part exists for the
    streamed shape only, d + 9 > 64)."""
    if split == "fp16x1" and d + 9 <= 64:
        pytest.skip("one FP16 part: streamed shape only")
    monkeypatch.setenv("SNN_TC_SPLIT", split)
    rng = np.random.default_rng(200 + d)
    centres = rng.uniform(-spread, spread, size=(6, d))
    lab = rng.integers(0, 6, size=4000)
    P = (centres[lab] + rng.standard_normal((4000, d))).astype(np.float32)
    Q = (centres[rng.integers(0, 6, size=500)] + rng.standard_normal((500, d))).astype(np.float32)
    R = float(np.sqrt(2.0 * d) * 0.8)
    want = {"bf16x2": snn.SNN_SPLIT_BF16X2, "bf16x3": snn.SNN_SPLIT_BF16X3, "fp16x2": snn.SNN_SPLIT_FP16X2,
            "fp16x1": snn.SNN_SPLIT_FP16X1}[split]
    for q in (None, Q):
        got = _run(snn, P, q, R, "bf16")
        assert got.stats["split_used"] == want
        assert_csr_equal(got, oracle.brute_radius(P, q, R), f"split={split} d={d}")


@pytest.mark.parametrize("d", [16, 40, 200])
def test_fp16_parts_scaling_and_small_values(snn, monkeypatch, d):
    """FP16 parts of rows scaled by 2^sigma: data far above and far below
    the FP16 range (sigma < 0 and sigma > 0), rows mixing magnitudes over
    thirty binades (parts below the FP16 normal range set to zero), and a
    radius far above the norms; every case equals the oracle bit for bit."""
    monkeypatch.setenv("SNN_TC_SPLIT", "fp16x2")
    rng = np.random.default_rng(300 + d)
    base = rng.standard_normal((3000, d))
    base[:, ::3] *= 2.0 ** -30                     # tiny columns next to unit ones
    base[::7] *= 2.0 ** -12                        # whole rows 4096x smaller
    for scale in (2.0 ** 40, 1.0, 2.0 ** -60):
        P = (base * scale).astype(np.float32)
        Q = (rng.standard_normal((400, d)) * scale).astype(np.float32)
        R = float(np.quantile(np.linalg.norm(P[:300, None, :] - P[None, :300, :], axis=2), 0.02))
        for q in (None, Q):
            got = _run(snn, P, q, R, "bf16")
            assert_csr_equal(got, oracle.brute_radius(P, q, R), f"d={d} scale={scale}")
    P = base.astype(np.float32)
    R = float(50.0 * np.sqrt(d))                    # every pair inside
    got = _run(snn, P, None, R, "bf16")
    ref = oracle.brute_radius(P, None, R)
    assert ref.nnz == 3000 * 3000
    assert_csr_equal(got, ref, f"d={d} large R")


@pytest.mark.parametrize("d", [64, 100, 784])
def test_fp16_single_part_scaling_and_small_values(snn, monkeypatch, d):
    """One FP16 part per row with its own power-of-two scale and the per-pair
    bound from the exact residual norms: data far above and far below the
    FP16 range, columns thirty binades below the others (rounded to zero and
    carried by the residual), rows 4096x smaller than the rest, a radius far
    above the norms (every pair inside), and out-of-sample queries of another
    scale; every case equals the oracle bit for bit."""
    monkeypatch.setenv("SNN_TC_SPLIT", "fp16x1")
    rng = np.random.default_rng(400 + d)
    base = rng.standard_normal((2500, d))
    base[:, ::3] *= 2.0 ** -30
    base[::7] *= 2.0 ** -12
    for scale in (2.0 ** 12, 1.0, 2.0 ** -40):
        P = (base * scale).astype(np.float32)
        Q = (rng.standard_normal((300, d)) * scale * 1.5).astype(np.float32)
        R = float(np.quantile(np.linalg.norm(P[:300, None, :] - P[None, :300, :], axis=2), 0.02))
        for q in (None, Q):
            got = _run(snn, P, q, R, "bf16")
            assert got.stats["split_used"] == snn.SNN_SPLIT_FP16X1, (d, scale)
            assert_csr_equal(got, oracle.brute_radius(P, q, R), f"d={d} scale={scale}")
    P = base.astype(np.float32)
    R = float(50.0 * np.sqrt(d))
    got = _run(snn, P, None, R, "bf16")
    ref = oracle.brute_radius(P, None, R)
    assert ref.nnz == 2500 * 2500
    assert_csr_equal(got, ref, f"d={d} large R")


@pytest.mark.parametrize("tiles", ["2", "1"])
def test_lowrank_img_single_part_default(snn, monkeypatch, tiles):
    """On the image-like data the automatic choice is one FP16 part per row
    (one MMA per k step); the set equals the oracle's and the survivors stay
    within a small multiple of the neighbour pairs, with two query tiles per
    work item (the default, 47 tiles: the last group half empty) and with
    one (SNN_H1_TILES=1)."""
    monkeypatch.setenv("SNN_H1_TILES", tiles)
    w = wl.lowrank_img(n=6007, sub=2000)
    got = _run(snn, w.P, None, w.R, "bf16")
    assert got.stats["split_used"] == snn.SNN_SPLIT_FP16X1
    assert got.stats["mma_flops_per_pair"] == 2 * 16 * (784 // 16 + 1)
    assert_csr_equal(got, oracle.brute_radius(w.P, None, w.R), "lowrank_img fp16x1")
    directed = 2 * got.stats["survivors"] - w.n
    assert directed <= 4 * got.nnz


@pytest.mark.parametrize("split", ["fp16x2", "fp16x1"])
def test_operand_cache_two_streams(snn, monkeypatch, split):
    """Queries of very different norm scales on one index from two streams,
    interleaved: the packed operands of the index are built once per kind
    and never replaced while queries may read them (the second stream waits
    for the packing of the first), and queries whose scaled coordinates would
    leave the FP16 range take BF16 parts for their call.  Every result
    equals the oracle."""
    monkeypatch.setenv("SNN_TC_SPLIT", split)
    d = 16 if split == "fp16x2" else 100
    rng = np.random.default_rng(501)
    P = rng.standard_normal((6000, d)).astype(np.float32)
    ix = snn.Index(_dev(P))
    Qs = [(rng.standard_normal((700, d)) * sc).astype(np.float32) for sc in (1.0, 40.0, 0.25)]
    Rs = [2.5, 60.0, 0.8]
    Qd = [_dev(Q) for Q in Qs]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for rep in range(2):
        for k, R in enumerate(Rs):
            st = streams[(k + rep) % 2]
            outs.append((k, ix.query(Qd[k], R, precision="bf16", stream=st, stats=True)))
    torch.cuda.synchronize()
    for k, got in outs:
        assert_csr_equal(got, oracle.brute_radius(P, Qs[k], Rs[k]), f"{split} set {k}")
    if split == "fp16x2":
        used = {k: got.stats["split_used"] for k, got in outs}
        assert used[0] == snn.SNN_SPLIT_FP16X2 and used[1] == snn.SNN_SPLIT_BF16X2
