"""GPU parity of cosine / angular search (Section 3's Euclidean reduction):
the row normalisation is bit-identical to the oracle's, and the neighbour
sets, their order and dist2 of the search on normalised rows equal the
oracle's for every precision."""
import math

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


def test_normalize_rows_bit_exact(snn):
    rng = np.random.default_rng(81)
    for d in (1, 3, 17, 100, 300, 784):
        X = (rng.standard_normal((1500, d)) * 10.0 ** rng.integers(-30, 31, (1500, 1))).astype(np.float32)
        X[::97] = 0.0                                   # zero rows stay zero
        X[5, 0] = 3.0e38                                # squares far beyond FP32
        if d > 1:
            X[7, :] = 1.0e-45                           # FP32 subnormal row
        got = snn.normalize_rows(_dev(X)).cpu().numpy()
        ref = oracle.normalize_rows(X)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), d
    # in place, and rows with a stride
    Xt = _dev(X)
    snn.normalize_rows(Xt, out=Xt)
    assert np.array_equal(Xt.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    W = _dev(np.hstack([X, np.full((X.shape[0], 5), 7.0, np.float32)]))[:, :X.shape[1]]
    assert np.array_equal(snn.normalize_rows(W).cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_cosine_self_join(snn, prec):
    w = wl.glove_like(n=4000, sub=2000)
    got = snn.cosine_radius_search(_dev(w.P), cos_dist=w.R, precision=prec)
    ref = oracle.cosine_radius(w.P, None, oracle.radius_for_cosine_distance(w.R))
    _check(got, ref, f"glove_like {prec}")
    # dist2 is twice the cosine distance: every returned pair is within 2 c
    assert float(got.dist2.max()) <= 2.0 * w.R * (1 + 1e-6)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_angular_out_of_sample(snn, prec):
    rng = np.random.default_rng(82)
    w = wl.glove_like(n=3000, d=64, clusters=30, sub=1500)
    Q = (w.P[rng.integers(0, w.n, 500)] + 0.2 * rng.standard_normal((500, w.d))).astype(np.float32)
    for deg in (20.0, 45.0, 70.0):
        t = math.cos(math.radians(deg))
        got = snn.cosine_radius_search(_dev(w.P), _dev(Q), cos_sim=t, precision=prec)
        ref = oracle.cosine_radius(w.P, Q, oracle.radius_for_cosine_similarity(t))
        _check(got, ref, f"angle {deg} {prec}")
