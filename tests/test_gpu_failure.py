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
