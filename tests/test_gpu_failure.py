"""Failure detection without faulting the GPU.

A test fault makes the tensor-core producer withhold its TMA loads; the
consumers' bounded mbarrier waits (about two seconds) must expire, the kernel
must free its tensor memory and return, the call must report SNN_ETIMEOUT, and
the CUDA context must stay usable for the next query.  Also the range guard:
data whose centred norms could overflow the FP32/BF16 scores is refused."""
import numpy as np
import pytest

import oracle

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


@pytest.mark.parametrize("d", [16, 100])
def test_stalled_pipeline_times_out_and_context_survives(snn, d):
    rng = np.random.default_rng(31)
    P = rng.standard_normal((3000, d)).astype(np.float32)
    R = float(np.sqrt(2.0 * d) * 0.7)
    ix = snn.Index(_dev(P))
    snn.test_inject(snn.SNN_FAULT_STALL_TC_PRODUCER)
    with pytest.raises(snn.SNNError) as e:
        ix.query(None, R, precision="bf16")
    assert e.value.status == snn.SNN_ETIMEOUT
    # the fault was one-shot and the context is intact
    ref = oracle.brute_radius(P, None, R)
    for prec in ("bf16", "fp32"):
        got = ix.query(None, R, precision=prec)
        assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets)
        assert np.array_equal(got.indices.cpu().numpy(), ref.ids)


def test_norm_range_guard(snn):
    P = np.random.default_rng(32).standard_normal((200, 3)).astype(np.float32) * np.float32(1e20)
    with pytest.raises(snn.SNNError) as e:
        snn.Index(_dev(P))
    assert e.value.status == snn.SNN_ENOTSUP
    # a far-away but tight cluster is fine: only centred norms matter
    Q = np.random.default_rng(33).standard_normal((200, 3)).astype(np.float32) + np.float32(1e6)
    ix = snn.Index(_dev(Q))
    got = ix.query(None, 1.0)
    assert np.array_equal(got.offsets.cpu().numpy(), oracle.brute_radius(Q, None, 1.0).offsets)
    far = (np.random.default_rng(34).standard_normal((10, 3)) * 1e20).astype(np.float32)
    with pytest.raises(snn.SNNError) as e:
        ix.query(_dev(far), 1.0)
    assert e.value.status == snn.SNN_ENOTSUP


@pytest.mark.parametrize("prec,oos", [("fp32", False), ("bf16", False), ("bf16", True)])
def test_survivor_overflow_rerun_gives_the_same_result(snn, prec, oos):
    """A one-entry survivor buffer overflows at once; the scorer counts
    without writing past the end and the query re-runs with the exact size."""
    rng = np.random.default_rng(35)
    P = rng.standard_normal((5000, 16)).astype(np.float32)
    Q = rng.standard_normal((700, 16)).astype(np.float32) if oos else None
    R = 3.0
    ix = snn.Index(_dev(P))
    snn.test_inject(snn.SNN_FAULT_SMALL_SURVIVOR_BUFFER)
    got = ix.query(None if Q is None else _dev(Q), R, precision=prec, stats=True)
    ref = oracle.brute_radius(P, Q, R)
    assert got.stats["survivors"] > 1
    assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets)
    assert np.array_equal(got.indices.cpu().numpy(), ref.ids)
    assert np.array_equal(got.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32))


def test_device_allocation_failure_is_reported_and_recovered(snn):
    """An injected allocation failure makes the call return SNN_ENOMEM; the
    call releases what it held, an index survives a failed insert unchanged,
    and the next calls succeed."""
    rng = np.random.default_rng(36)
    P = rng.standard_normal((3000, 8)).astype(np.float32)
    R = 1.5
    try:
        snn.test_inject(snn.SNN_FAULT_DEVICE_ALLOC)
        with pytest.raises(snn.SNNError) as e:
            snn.Index(_dev(P))
        assert e.value.status == snn.SNN_ENOMEM
        ix = snn.Index(_dev(P))
        ref = oracle.brute_radius(P, None, R)
        snn.test_inject(snn.SNN_FAULT_DEVICE_ALLOC)
        with pytest.raises(snn.SNNError) as e:
            ix.query(None, R, precision="bf16")
        assert e.value.status == snn.SNN_ENOMEM
        got = ix.query(None, R, precision="bf16")
        assert np.array_equal(got.indices.cpu().numpy(), ref.ids)
        # a failed insert leaves the index as it was
        snn.test_inject(snn.SNN_FAULT_DEVICE_ALLOC)
        extra = rng.standard_normal((500, 8)).astype(np.float32)
        with pytest.raises(snn.SNNError) as e:
            ix.insert(_dev(extra))
        assert e.value.status == snn.SNN_ENOMEM
        got = ix.query(None, R, precision="fp32")
        assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets)
        assert np.array_equal(got.indices.cpu().numpy(), ref.ids)
        ix.insert(_dev(extra))
        both = np.concatenate([P, extra])
        got = ix.query(None, R, precision="fp32")
        assert np.array_equal(got.indices.cpu().numpy(), oracle.brute_radius(both, None, R).ids)
    finally:
        snn.test_inject(0)
