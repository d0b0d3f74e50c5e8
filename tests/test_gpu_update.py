"""Streaming index updates: after inserts and deletes, every query equals the
FP64 oracle on the updated point set (rows appended, or erased with the rest
renumbered), for every precision, although the index keeps its original
centre and direction."""
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


def _check(got, ref, what):
    assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets), what
    assert np.array_equal(got.indices.cpu().numpy(), ref.ids), what
    assert np.array_equal(got.dist2.cpu().numpy().view(np.uint32), ref.dist2.view(np.uint32)), what


def _mixture(rng, n, d, centres, std=1.0):
    return (centres[rng.integers(0, len(centres), n)] + std * rng.standard_normal((n, d))).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_inserts_match_a_fresh_build(snn, prec):
    rng = np.random.default_rng(91)
    d = 12
    centres = rng.uniform(-6, 6, (6, d))
    P = _mixture(rng, 3000, d, centres)
    ix = snn.Index(_dev(P))
    R = 1.7
    # new points: the same mixture, a cluster elsewhere (beyond the score
    # range and across the original direction), duplicates of old points
    far = _mixture(rng, 700, d, rng.uniform(20, 30, (2, d)))
    dup = P[rng.integers(0, 3000, 300)]
    Q = _mixture(rng, 400, d, centres)
    for add in (_mixture(rng, 1000, d, centres), far, dup):
        ix.insert(_dev(add))
        P = np.vstack([P, add])
        assert ix.n == P.shape[0]
        _check(ix.query(None, R, precision=prec), oracle.brute_radius(P, None, R), f"self-join n={P.shape[0]}")
        _check(ix.query(_dev(Q), R, precision=prec), oracle.brute_radius(P, Q, R), f"queries n={P.shape[0]}")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_deletes_renumber_the_rest(snn, prec):
    rng = np.random.default_rng(92)
    d = 70
    centres = rng.uniform(-3, 3, (5, d))
    P = _mixture(rng, 2500, d, centres)
    ix = snn.Index(_dev(P))
    R = float(np.sqrt(2.0 * d) * 0.8)
    for cut in (rng.choice(P.shape[0], 400, replace=False), np.array([0, 0, 5, P.shape[0] - 1 - 400])):
        ix.delete(cut)
        P = np.delete(P, np.unique(cut), axis=0)
        assert ix.n == P.shape[0]
        _check(ix.query(None, R, precision=prec), oracle.brute_radius(P, None, R), f"after delete n={P.shape[0]}")
    # insert after delete, then delete again
    add = _mixture(rng, 600, d, centres)
    ix.insert(_dev(add))
    P = np.vstack([P, add])
    ix.delete(np.arange(100, 300))
    P = np.delete(P, np.arange(100, 300), axis=0)
    _check(ix.query(None, R, precision=prec), oracle.brute_radius(P, None, R), "insert then delete")


def test_invalid_updates_leave_the_index_unchanged(snn):
    rng = np.random.default_rng(93)
    P = rng.standard_normal((800, 5)).astype(np.float32)
    ix = snn.Index(_dev(P))
    ref = oracle.brute_radius(P, None, 0.9)
    bad = rng.standard_normal((10, 5)).astype(np.float32)
    bad[3, 2] = np.nan
    with pytest.raises(snn.SNNError) as e:
        ix.insert(_dev(bad))
    assert e.value.status == snn.SNN_EINVAL
    with pytest.raises(snn.SNNError):
        ix.delete([5, 800])
    with pytest.raises(snn.SNNError):
        ix.delete(np.arange(800))
    ix.n = 800
    _check(ix.query(None, 0.9, precision="bf16"), ref, "unchanged")


def test_update_of_a_batched_index(snn):
    rng = np.random.default_rng(94)
    sets = [rng.standard_normal((n, d)).astype(np.float32) for n, d in ((900, 3), (1200, 8), (700, 32))]
    idx = snn.build_batch([_dev(x) for x in sets])
    add = rng.standard_normal((300, 8)).astype(np.float32) * 2
    idx[1].insert(_dev(add))
    idx[2].delete(np.arange(0, 700, 3))
    want = [sets[0], np.vstack([sets[1], add]), np.delete(sets[2], np.arange(0, 700, 3), axis=0)]
    for t, (ix, P) in enumerate(zip(idx, want)):
        _check(ix.query(None, 1.1, precision="bf16"), oracle.brute_radius(P, None, 1.1), f"set {t}")


def test_index_save_load_round_trip(snn):
    """An index restored from its saved image answers every query exactly as
    the saved one did (and as the oracle does), also after updates."""
    rng = np.random.default_rng(71)
    P = rng.standard_normal((6000, 20)).astype(np.float32)
    R = 3.2
    ix = snn.Index(_dev(P))
    image = ix.save()
    ix2 = snn.Index.load(image)
    assert (ix2.n, ix2.d) == (6000, 20)
    ref = oracle.brute_radius(P, None, R)
    for prec in ("fp32", "bf16"):
        a = ix.query(None, R, precision=prec)
        b = ix2.query(None, R, precision=prec)
        assert np.array_equal(b.offsets.cpu().numpy(), ref.offsets)
        assert np.array_equal(b.indices.cpu().numpy(), ref.ids)
        assert np.array_equal(b.dist2.cpu().numpy().view(np.uint32), a.dist2.cpu().numpy().view(np.uint32))
    # updates on the restored index, then a second round trip
    extra = rng.standard_normal((700, 20)).astype(np.float32)
    ix2.insert(_dev(extra))
    ix2.delete(np.arange(0, 6700, 7, dtype=np.int32))
    keep = np.ones(6700, dtype=bool)
    keep[::7] = False
    cur = np.concatenate([P, extra])[keep]
    ix3 = snn.Index.load(ix2.save())
    Q = rng.standard_normal((500, 20)).astype(np.float32)
    for idx in (ix2, ix3):
        got = idx.query(_dev(Q), R, precision="bf16")
        ref = oracle.brute_radius(cur, Q, R)
        assert np.array_equal(got.offsets.cpu().numpy(), ref.offsets)
        assert np.array_equal(got.indices.cpu().numpy(), ref.ids)
    # a byte image is plain data: saving the restored index gives the same bytes
    assert ix3.save() == ix2.save()
