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
