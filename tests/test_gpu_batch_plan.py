"""GPU parity of the batched index build and of the graph-capturable batched
query plan (ragged batches of independent sets) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2212_07679_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_07679_gb300 import snn as mod
    return mod


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _eq(got, ref, what):
    off = got.offsets.cpu().numpy()
    assert np.array_equal(off, ref.offsets), what
    assert np.array_equal(got.indices.cpu().numpy(), ref.ids), what
    assert np.array_equal(got.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32)), what


def _sets():
    sets = wl.ragged_batch(sets=10, n_lo=400, n_hi=5000, seed=123)
    rng = np.random.default_rng(5)
    # extra shapes: d = 17 and 64, a single point, exact integer ties
    sets.append(wl.Workload("d17", rng.standard_normal((900, 17)).astype(np.float32), None, 2.5))
    sets.append(wl.Workload("d64", rng.standard_normal((700, 64)).astype(np.float32), None, 9.0))
    sets.append(wl.Workload("n1", np.array([[1.0, 2.0]], np.float32), None, 0.0))
    grid = np.stack(np.meshgrid(np.arange(9), np.arange(9)), -1).reshape(-1, 2).astype(np.float32)
    sets.append(wl.Workload("grid", grid, grid[::7].copy(), 1.0))
    return sets


def test_build_batch_matches_oracle(snn):
    sets = _sets()
    idx = snn.build_batch([_dev(s.P) for s in sets])
    for s, ix in zip(sets, idx):
        v = ix.view()
        alpha = v["alpha"].cpu().numpy()
        order = v["order"].cpu().numpy()
        assert np.all(np.diff(alpha) >= 0), s.name
        assert np.array_equal(np.sort(order), np.arange(s.P.shape[0])), s.name
        assert np.array_equal(v["points"].cpu().numpy(), s.P[order]), s.name
        c = v["centre"].cpu().numpy().astype(np.float64)
        a64 = (s.P[order].astype(np.float64) - c) @ v["v1"].cpu().numpy()
        assert np.max(np.abs(alpha - a64)) <= v["alpha_err"], s.name
        got = ix.query(None if s.Q is None else _dev(s.Q), s.R)
        _eq(got, oracle.brute_radius(s.P, s.Q, s.R), s.name)


def test_build_batch_rejects_bad_sets(snn):
    P = np.zeros((10, 3), np.float32)
    P[4, 1] = np.nan
    with pytest.raises(snn.SNNError) as e:
        snn.build_batch([_dev(np.ones((5, 2))), _dev(P)])
    assert e.value.status == snn.SNN_EINVAL
    with pytest.raises(snn.SNNError):
        snn.build_batch([_dev(np.ones((5, 65)))])      # d > 64


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_plan_run_graph_and_tune(snn, prec):
    sets = _sets()
    idx = snn.build_batch([_dev(s.P) for s in sets])
    ms = [None if s.Q is None else s.Q.shape[0] for s in sets]
    plan = snn.BatchPlan(idx, ms, [s.R for s in sets], precision=prec,
                         survivor_capacity=1 << 22, nnz_capacity=1 << 22)
    for t, s in enumerate(sets):
        if s.Q is not None:
            plan.queries(t).copy_(_dev(s.Q))
    refs = [oracle.brute_radius(s.P, s.Q, s.R) for s in sets]
    plan.run()
    for s, got, ref in zip(sets, plan.result(), refs):
        _eq(got, ref, f"run {s.name}")
    # graph replay, twice, with new query values of the same shape
    rng = np.random.default_rng(17)
    for rep in range(2):
        newQ = {}
        for t, s in enumerate(sets):
            if s.Q is not None:
                q = (s.Q + rng.normal(0, 0.3, s.Q.shape)).astype(np.float32)
                newQ[t] = q
                plan.queries(t).copy_(_dev(q))
        plan.launch_graph()
        for t, (s, got) in enumerate(zip(sets, plan.result())):
            _eq(got, oracle.brute_radius(s.P, newQ.get(t), s.R), f"graph {rep} {s.name}")
    cpi, ctas, ms_best = plan.tune()
    assert cpi in (4, 8, 16, 32) and ctas in (1, 2) and ms_best > 0
    plan.launch_graph()
    for t, (s, got) in enumerate(zip(sets, plan.result())):
        _eq(got, oracle.brute_radius(s.P, newQ.get(t), s.R), f"tuned {s.name}")
    plan.close()


def test_plan_reports_overflow_and_nan(snn):
    sets = _sets()[:4]
    idx = snn.build_batch([_dev(s.P) for s in sets])
    ms = [None if s.Q is None else s.Q.shape[0] for s in sets]
    small = snn.BatchPlan(idx, ms, [s.R for s in sets], survivor_capacity=1024, nnz_capacity=1024)
    for t, s in enumerate(sets):
        if s.Q is not None:
            small.queries(t).copy_(_dev(s.Q))
    small.run()
    with pytest.raises(snn.SNNError) as e:
        small.result()
    assert e.value.status == snn.SNN_EOVERFLOW
    # NaN in a query set
    plan = snn.BatchPlan(idx, ms, [s.R for s in sets], survivor_capacity=1 << 22,
                         nnz_capacity=1 << 22)
    t = next(t for t, s in enumerate(sets) if s.Q is not None)
    for u, s in enumerate(sets):
        if s.Q is not None:
            plan.queries(u).copy_(_dev(s.Q))
    q = plan.queries(t)
    q[0, 0] = float("nan")
    plan.run()
    with pytest.raises(snn.SNNError) as e:
        plan.result()
    assert e.value.status == snn.SNN_EINVAL
    # the same plan recovers with clean queries
    plan.queries(t).copy_(_dev(sets[t].Q))
    plan.run()
    for s, got in zip(sets, plan.result()):
        _eq(got, oracle.brute_radius(s.P, s.Q, s.R), s.name)


def test_plan_set_queries_one_launch(snn):
    """set_queries copies every out-of-sample set's rows (contiguous or with
    a row stride) in one launch: the same result as per-set copies; a wrong
    shape or a missing set is refused."""
    sets = _sets()
    idx = snn.build_batch([_dev(s.P) for s in sets])
    ms = [None if s.Q is None else s.Q.shape[0] for s in sets]
    plan = snn.BatchPlan(idx, ms, [s.R for s in sets], survivor_capacity=1 << 22, nnz_capacity=1 << 22)
    qs = []
    for s in sets:
        if s.Q is None:
            qs.append(None)
            continue
        wide = torch.zeros((s.Q.shape[0], s.Q.shape[1] + 5), dtype=torch.float32, device="cuda")
        wide[:, :s.Q.shape[1]] = _dev(s.Q)
        qs.append(wide[:, :s.Q.shape[1]])          # row stride d + 5
    launches = snn.launch_count()
    plan.set_queries(qs)
    assert snn.launch_count() - launches == 1
    for t, s in enumerate(sets):
        if s.Q is not None:
            assert torch.equal(plan.queries(t), _dev(s.Q)), t
    plan.run()
    copies = plan.result()
    views = plan.result(copy=False)              # per-set views, made on access
    assert len(views) == len(sets)
    for s, got, v in zip(sets, copies, views):
        _eq(got, oracle.brute_radius(s.P, s.Q, s.R), s.name)
        assert torch.equal(v.offsets, got.offsets) and torch.equal(v.indices, got.indices), s.name
        assert torch.equal(v.dist2, got.dist2), s.name
    assert torch.equal(views[-1].indices, copies[-1].indices) and len(views[1:3]) == 2
    t = next(t for t, s in enumerate(sets) if s.Q is not None)
    bad = list(qs)
    bad[t] = qs[t][:-1]
    with pytest.raises(ValueError):
        plan.set_queries(bad)
    with pytest.raises(ValueError):
        plan.set_queries(qs[:-1])
    plan.close()


def _plan(snn, sets, prec, cap=1 << 22):
    idx = snn.build_batch([_dev(s.P) for s in sets])
    ms = [None if s.Q is None else s.Q.shape[0] for s in sets]
    plan = snn.BatchPlan(idx, ms, [s.R for s in sets], precision=prec, survivor_capacity=cap,
                         nnz_capacity=cap)
    for t, s in enumerate(sets):
        if s.Q is not None:
            plan.queries(t).copy_(_dev(s.Q))
    return idx, plan


def test_plan_tensor_core_groups(snn, tmp_path, monkeypatch):
    """With 16-bit precision the out-of-sample sets of d <= 48 are scored by
    tensor-core groups (one per rounded width); sets of several query tiles
    with odd tile counts (padded tile pairs), a self-join set and a d = 64
    set left to the FP32 scorer.  Every group choice the tuner tries ends in
    the oracle's result; a tuned choice is stored in the SNN_TUNE_CACHE file
    and a second plan of the same shape takes it from there."""
    rng = np.random.default_rng(41)
    sets = []
    for d, n, m in [(2, 3000, 700), (3, 2500, 300), (8, 4000, 390), (32, 3500, 520), (40, 2000, 260),
                    (16, 1500, 129), (24, 1800, 1)]:
        c = rng.uniform(-8, 8, size=(5, d))
        P = (c[rng.integers(0, 5, n)] + rng.standard_normal((n, d))).astype(np.float32)
        Q = (c[rng.integers(0, 5, m)] + rng.standard_normal((m, d))).astype(np.float32)
        R = float(np.quantile(np.linalg.norm(P[:300, None] - P[None, :300], axis=2), 0.01))
        sets.append(wl.Workload(f"d{d}", P, Q, R))
    sets.append(wl.Workload("self", rng.standard_normal((900, 8)).astype(np.float32), None, 0.6))
    sets.append(wl.Workload("d64", rng.standard_normal((600, 64)).astype(np.float32),
                            rng.standard_normal((70, 64)).astype(np.float32), 9.0))
    refs = [oracle.brute_radius(s.P, s.Q, s.R) for s in sets]
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("SNN_TUNE_CACHE", str(cache))
    idx, plan = _plan(snn, sets, "bf16")
    cfg = plan.config()
    assert cfg["tc_groups"] == 3 and cfg["tc_mask"] == 7
    plan.run()
    for s, got, ref in zip(sets, plan.result(), refs):
        _eq(got, ref, f"tc run {s.name}")
    cpi, ctas, ms_best = plan.tune()
    assert ms_best > 0 and not plan.config()["from_cache"]
    plan.launch_graph()
    for s, got, ref in zip(sets, plan.result(), refs):
        _eq(got, ref, f"tuned {s.name}")
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"tc_mask"' in lines[0]
    plan.close()
    idx2, plan2 = _plan(snn, sets, "bf16")
    cpi2, ctas2, ms2 = plan2.tune()
    cfg2 = plan2.config()
    assert cfg2["from_cache"] and ms2 == 0 and (cpi2, ctas2) == (cpi, ctas)
    plan2.run()
    for s, got, ref in zip(sets, plan2.result(), refs):
        _eq(got, ref, f"cached {s.name}")
    plan2.close()


def test_plan_tensor_core_query_range(snn):
    """A query far beyond the FP16 range of its set's scaled operands is
    reported (SNN_ENOTSUP) instead of scored; the FP32 plan answers it."""
    rng = np.random.default_rng(42)
    P = rng.standard_normal((2000, 8)).astype(np.float32)
    Q = rng.standard_normal((200, 8)).astype(np.float32)
    Q[17] *= 1e4
    sets = [wl.Workload("far", P, Q, 1.0)]
    _, plan = _plan(snn, sets, "bf16")
    plan.run()
    with pytest.raises(snn.SNNError) as e:
        plan.result()
    assert e.value.status == snn.SNN_ENOTSUP
    plan.close()
    _, plan = _plan(snn, sets, "fp32")
    plan.run()
    _eq(plan.result()[0], oracle.brute_radius(P, Q, 1.0), "fp32 far")
    plan.close()
