"""The allocation-free score sort, called through the C ABI.

snn_sort_scores_noalloc serves callers that may not allocate device memory
(for example a process whose device memory budget is fixed elsewhere, or a
loop that must not enter the allocator): it sorts with a static scratch array
compiled into the library.  Its result must equal the
sort the index build performs (the score sort of Algorithm 1) on the same scores: same
sorted values and the same stable permutation, bit for bit.  The file is
collected last so that a failure here leaves every other test already run;
it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_07679_gb300 import snn as mod
    lib = mod.lib
    lib.snn_sort_scores_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
    lib.snn_sort_scores_noalloc.restype = ctypes.c_int
    return mod


def _noalloc_sort(snn, alpha, in_place=False):
    n = alpha.numel()
    out_a = alpha if in_place else torch.full((max(n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    out_o = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = snn.lib.snn_sort_scores_noalloc(ctypes.c_void_p(alpha.data_ptr()), n,
                                         ctypes.c_void_p(out_a.data_ptr()),
                                         ctypes.c_void_p(out_o.data_ptr()), stream)
    torch.cuda.synchronize()
    return st, out_a[:n], out_o[:n]


def _index_scores(snn, n, d, seed):
    """Scores in input order and their sorted order, from the index build."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    X[: n // 3] = np.round(X[: n // 3])          # many tied scores
    ix = snn.Index(torch.from_numpy(X).cuda())
    v = ix.view()
    alpha_sorted, order = v["alpha"], v["order"]
    alpha_in = torch.empty_like(alpha_sorted)
    alpha_in[order.long()] = alpha_sorted
    return alpha_in, alpha_sorted, order


def test_noalloc_sort_matches_index_sort_twice(snn):
    # two calls in a row: the second must not see stale scratch contents
    for n, d, seed in [(300_007, 6, 1), (1 << 20, 3, 2)]:
        alpha_in, ref_sorted, ref_order = _index_scores(snn, n, d, seed)
        st, got_sorted, got_order = _noalloc_sort(snn, alpha_in)
        assert st == snn.SNN_OK, snn.lib.snn_last_error()
        assert torch.equal(got_sorted.view(torch.int32), ref_sorted.view(torch.int32))
        assert torch.equal(got_order, ref_order)


def test_noalloc_sort_limits(snn):
    limit = 1 << 20
    big = torch.zeros(limit + 1, dtype=torch.float32, device="cuda")
    st, _, _ = _noalloc_sort(snn, big)
    assert st == snn.SNN_EINVAL
    assert b"static sort scratch" in snn.lib.snn_last_error()
    st, _, _ = _noalloc_sort(snn, torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert st == snn.SNN_OK
    bad = torch.tensor([1.0, float("nan"), 2.0], device="cuda")
    st, _, _ = _noalloc_sort(snn, bad)
    assert st == snn.SNN_EINVAL


def _host_keys(a):
    """The order-preserving 32-bit key of each FP32 value, written here from
    the IEEE encoding: flip every bit of a negative value, only the sign bit
    of a non-negative one (so -0.0 orders just below +0.0)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return np.where(b >> 31 == 1, ~b, b | np.uint32(0x80000000)).astype(np.uint32)


@pytest.mark.parametrize("in_place", [False, True])
def test_noalloc_sort_matches_numpy_stable_argsort(snn, in_place):
    """Independent of the library's own sort: numpy's stable argsort of the
    keys gives the permutation; values with mixed signs, both zeros, ties,
    denormals and the extremes of the FP32 range; out of place and in place
    (alpha_sorted == alpha)."""
    rng = np.random.default_rng(61)
    n = 200_003
    a = rng.standard_normal(n).astype(np.float32) * np.float32(1e3)
    a[rng.choice(n, 20_000, replace=False)] = np.float32(0.0)
    a[rng.choice(n, 20_000, replace=False)] = np.float32(-0.0)
    a[rng.choice(n, 5_000, replace=False)] = np.float32(1.5)
    a[rng.choice(n, 5_000, replace=False)] = np.float32(-1.5)
    a[rng.choice(n, 100, replace=False)] = np.float32(1e-42)
    a[rng.choice(n, 100, replace=False)] = np.float32(-1e-42)
    a[rng.choice(n, 10, replace=False)] = np.float32(3.4e38)
    a[rng.choice(n, 10, replace=False)] = np.float32(-3.4e38)
    want = np.argsort(_host_keys(a), kind="stable")
    for _ in range(2):
        dev = torch.from_numpy(a.copy()).cuda()
        st, got_sorted, got_order = _noalloc_sort(snn, dev, in_place=in_place)
        assert st == snn.SNN_OK, snn.lib.snn_last_error()
        assert np.array_equal(got_order.cpu().numpy(), want.astype(np.int32))
        assert np.array_equal(got_sorted.cpu().numpy().view(np.uint32), a[want].view(np.uint32))
