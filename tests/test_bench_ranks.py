"""The benchmark's multi-rank host logic on CPU: two gloo ranks (127.0.0.1),
each with its own timed total; every rank must see the job time as the
largest total, and the whole-job rate counts the units of every replica."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, totals, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        ms = bench.job_max_ms(totals[rank], world)
        out[rank] = ms
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks():
    world = 2
    totals = [12.5, 40.25]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, totals, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert out[0] == out[1] == max(totals)


def test_single_rank_and_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_max_ms(7.0, 1) == 7.0
    # two replicas of 1,000 queries in 10 ms: 200,000 queries/s for the job
    assert bench.whole_job_rate(1000, 2, 10.0) == pytest.approx(2.0e5)


def test_scorer_traffic_is_tied_to_the_scorer_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from a capture of one scorer build: it is
    reported for the captured workloads while the scorer sources hash to the
    recorded value, and null for any other workload or source."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import hashlib
    h = hashlib.sha256()
    for f in bench.SCORER_SOURCES:
        with open(os.path.join(ROOT, "paper_2212_07679_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    expect = (bench.SCORER_TRAFFIC[("gmm_aniso", 1000000, "bf16")]
              if h.hexdigest()[:16] == bench.SCORER_TRAFFIC["sha"] else None)
    assert bench.scorer_traffic("gmm_aniso", 1000000, "bf16") == expect
    assert bench.scorer_traffic("gmm_aniso", 12345, "bf16") is None
    assert bench.scorer_traffic("glove_like", 200000, "bf16") is None
    monkeypatch.setitem(bench.SCORER_TRAFFIC, "sha", "0000000000000000")
    assert bench.scorer_traffic("gmm_aniso", 1000000, "bf16") is None


def test_timed_regions_run_without_the_cyclic_collector():
    import gc
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert gc.isenabled()
    with bench.no_gc():
        assert not gc.isenabled()
    assert gc.isenabled()
