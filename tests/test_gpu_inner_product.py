"""GPU parity of the inner-product threshold search: the ids and the FP64
dot products (rounded to FP32) equal the oracle's bit for bit, whatever the
precision of the Euclidean pruning stage."""
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


def _check(got, ref, what):
    assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets), what
    assert np.array_equal(got.indices.cpu().numpy(), ref.ids), what
    assert np.array_equal(got.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32)), what


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_random_thresholds(snn, prec):
    rng = np.random.default_rng(101)
    P = (rng.standard_normal((3000, 12)) * rng.lognormal(0, 0.5, (3000, 1))).astype(np.float32)
    Q = rng.standard_normal((300, 12)).astype(np.float32)
    for tau in (9.0, 4.0, 0.0, -2.0):
        got = snn.inner_product_search(_dev(P), _dev(Q), tau, precision=prec, stats=True)
        _check(got, oracle.brute_inner_product(P, Q, tau), f"tau={tau}")
        st = got.stats
        assert st["candidates"] >= st["nnz"] == got.nnz


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_word_vectors(snn, prec):
    w = wl.mips_like(n=4000, m=400, sub=1000)
    got = snn.inner_product_search(_dev(w.P), _dev(w.Q), w.R, precision=prec)
    _check(got, oracle.brute_inner_product(w.P, w.Q, w.R), "mips_like")
    assert got.nnz > 0


def test_edge_cases(snn):
    rng = np.random.default_rng(102)
    # integer vectors: many dot products equal tau exactly (the FP64 loop decides)
    P = rng.integers(-3, 4, (1500, 9)).astype(np.float32)
    Q = rng.integers(-3, 4, (200, 9)).astype(np.float32)
    Q[0] = 0.0                                               # D = 0 for every point
    got = snn.inner_product_search(_dev(P), _dev(Q), 6.0, precision="bf16", stats=True)
    _check(got, oracle.brute_inner_product(P, Q, 6.0), "integer ties")
    assert got.stats["exact_fp64"] > 0
    _check(snn.inner_product_search(_dev(P), _dev(Q), 0.0), oracle.brute_inner_product(P, Q, 0.0), "tau 0")
    # nothing reaches the threshold / everything does
    assert snn.inner_product_search(_dev(P), _dev(Q), 1e6).nnz == 0
    Ps, Qs = P[:400], Q[:30]
    _check(snn.inner_product_search(_dev(Ps), _dev(Qs), -1e6), oracle.brute_inner_product(Ps, Qs, -1e6), "all")
    # rows of very different magnitudes, and d > 128 (32 lanes per pair)
    P2 = (rng.standard_normal((800, 150)) * 10.0 ** rng.integers(-4, 5, (800, 1))).astype(np.float32)
    Q2 = rng.standard_normal((60, 150)).astype(np.float32)
    for tau in (50.0, 0.5):
        _check(snn.inner_product_search(_dev(P2), _dev(Q2), tau), oracle.brute_inner_product(P2, Q2, tau),
               f"magnitudes tau={tau}")


@pytest.mark.parametrize("prec,d", [("fp32", 10), ("bf16", 10), ("bf16", 100), ("fp8", 100)])
def test_query_radius_each(snn, prec, d):
    """One radius per query: each row equals the oracle run with that radius."""
    rng = np.random.default_rng(103)
    scale = 2.0 if d == 10 else 0.4
    P = (rng.standard_normal((4000, d)) * scale).astype(np.float32)
    Q = (rng.standard_normal((600, d)) * scale).astype(np.float32)
    R = rng.uniform(0.0, 3.0 if d == 10 else 6.0, 600)
    R[::50] = 0.0
    got = snn.Index(_dev(P)).query_each(_dev(Q), R, precision=prec, stats=True)
    assert got.stats["precision_used"] == {"fp32": 0, "bf16": 1, "fp8": 2}[prec]
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    for t in range(0, 600, 7):
        ref = oracle.brute_radius(P, Q[t:t + 1], float(R[t]))
        a, b = off[t], off[t + 1]
        assert np.array_equal(idx[a:b], ref.ids), t
        assert np.array_equal(d2[a:b].view(np.uint32), ref.dist2.view(np.uint32)), t
    with pytest.raises(snn.SNNError):
        snn.Index(_dev(P)).query_each(_dev(Q), -R)
