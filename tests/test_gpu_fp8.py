"""GPU parity of the FP8 e4m3 rejection variant against the FP64 oracle.

FP8 only rejects pairs (its per-pair bound is built from the measured norms
of each row's e4m3 parts and exact residual), so the neighbour sets, their
order and the squared distances must equal the oracle's bit for bit, for
every product count (3 and 4: two e4m3 parts; 6: three parts)."""
import numpy as np
import pytest

import oracle
from paper_2212_07679_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRODUCTS = ["3", "4", "6"]


@pytest.fixture(scope="module")
def snn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_07679_gb300 import snn as mod
    return mod


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _check(got, P, Q, R, what):
    ref = oracle.brute_radius(P, Q, R)
    off = got.offsets.cpu().numpy()
    assert np.array_equal(off, ref.offsets), what
    assert np.array_equal(got.indices.cpu().numpy(), ref.ids), what
    assert np.array_equal(got.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32)), what


def _fp8(snn, P, Q, R):
    ix = snn.Index(_dev(P))
    return ix.query(None if Q is None else _dev(Q), R, precision="fp8", stats=True)


@pytest.mark.parametrize("products", PRODUCTS)
def test_fp8_lowrank_img_self_join(snn, monkeypatch, products):
    monkeypatch.setenv("SNN_FP8_PRODUCTS", products)
    w = wl.lowrank_img(n=3001, sub=1500)
    got = _fp8(snn, w.P, None, w.R)
    _check(got, w.P, None, w.R, f"lowrank_img products={products}")
    st = got.stats
    assert st["precision_used"] == 2
    # the symmetric self-join counts each unordered survivor once, itself included
    assert 2 * st["survivors"] - w.n >= st["nnz"] == got.nnz
    np_ = int(products)
    assert st["mma_flops_per_pair"] == 2 * 32 * np_ * 25 + 32


@pytest.mark.parametrize("products", PRODUCTS)
def test_fp8_out_of_sample_and_ragged_d(snn, monkeypatch, products):
    monkeypatch.setenv("SNN_FP8_PRODUCTS", products)
    rng = np.random.default_rng(61)
    for d in (57, 100, 161):
        centres = rng.uniform(-3, 3, size=(5, d))
        P = (centres[rng.integers(0, 5, 2600)] + rng.standard_normal((2600, d))).astype(np.float32)
        Q = (centres[rng.integers(0, 5, 333)] + rng.standard_normal((333, d))).astype(np.float32)
        for R in (0.0, float(np.sqrt(2.0 * d) * 0.85)):
            got = _fp8(snn, P, Q, R)
            _check(got, P, Q, R, f"oos d={d} R={R}")
            assert got.stats["precision_used"] == 2


@pytest.mark.parametrize("products", PRODUCTS)
def test_fp8_scaling_edge_cases(snn, monkeypatch, products):
    """Rows whose per-row scale hits the clamp or whose elements fall into the
    e4m3 subnormal range, rows equal to the mean (scale 0 rows), large common
    offsets and exact ties on R^2."""
    monkeypatch.setenv("SNN_FP8_PRODUCTS", products)
    rng = np.random.default_rng(62)
    cases = []
    same = np.repeat(rng.standard_normal((1, 96)).astype(np.float32), 300, axis=0)
    cases.append(("identical d=96", same, None, 0.0))
    off = (rng.standard_normal((1000, 80)) * 0.5 + 3e3).astype(np.float32)
    cases.append(("offset d=80", off, None, 3.0))
    # (each set below holds every row and its negation, so the mean is 0 and
    # the centred rows keep their magnitudes)
    # one large coordinate next to tiny ones: most e4m3 parts subnormal
    spiky = (rng.standard_normal((1500, 64)) * 1e-3).astype(np.float32)
    spiky[np.arange(1500), rng.integers(0, 64, 1500)] += rng.choice([-50.0, 50.0], 1500)
    spiky = np.vstack([spiky, -spiky])
    cases.append(("spiky d=64", spiky, None, 0.011))
    # rows at many magnitudes (scales clamped at 2^24 for the smallest)
    mags = (rng.standard_normal((1200, 70)) * 10.0 ** rng.integers(-12, 3, (1200, 1))).astype(np.float32)
    mags = np.vstack([mags, -mags])
    cases.append(("magnitudes d=70", mags, None, 1e-3))
    cases.append(("magnitudes d=70 R=5", mags, None, 5.0))
    binary = rng.integers(0, 2, (500, 200)).astype(np.float32)
    cases.append(("binary d=200 ties", binary, None, 10.0))
    for name, P, Q, R in cases:
        got = _fp8(snn, P, Q, R)
        _check(got, P, Q, R, name)
        assert got.stats["precision_used"] == 2, name


def test_fp8_falls_back_to_bf16(snn):
    rng = np.random.default_rng(63)
    P = rng.standard_normal((3000, 40)).astype(np.float32)
    got = _fp8(snn, P, None, 7.0)
    _check(got, P, None, 7.0, "d=40")
    assert got.stats["precision_used"] == 1
    big = (rng.standard_normal((800, 90)) * 3e6).astype(np.float32)
    got = _fp8(snn, big, None, 2e7)
    _check(got, big, None, 2e7, "norms above 2^20")
    assert got.stats["precision_used"] == 1


@pytest.mark.slow
def test_fp8_full_size_lowrank_img_sampled(snn):
    w = wl.lowrank_img()
    got = snn.Index(_dev(w.P)).query(None, w.R, precision="fp8", stats=True)
    assert got.stats["precision_used"] == 2
    rows = np.random.default_rng(64).choice(w.n, size=24, replace=False)
    off = got.offsets.cpu().numpy()
    idx = got.indices.cpu().numpy()
    d2 = got.dist2.cpu().numpy()
    ref = oracle.brute_radius(w.P, w.P[rows], w.R)
    for t, r in enumerate(rows):
        ri, rd = ref.row(t)
        a, b = off[r], off[r + 1]
        assert np.array_equal(idx[a:b], ri), r
        assert np.array_equal(d2[a:b].view(np.uint32), rd.view(np.uint32)), r
    rowid = np.repeat(np.arange(w.n, dtype=np.int64), np.diff(off))
    ids = idx.astype(np.int64)
    assert np.array_equal(np.sort(rowid * w.n + ids), np.sort(ids * w.n + rowid))
