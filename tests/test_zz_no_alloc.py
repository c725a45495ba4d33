"""ts_enumerate_noalloc: the sweep entry point for callers that cannot
allocate device memory at call time.  Its results, read from the caller's
output buffers, must equal those of ts_enumerate + ts_hist_read on the same
range, on two calls in a row (the second call reuses the static scratch the
first one left behind).  Kept in a file of its own, collected last."""
import collections
import ctypes

import numpy as np
import pytest

import tcurve_inputs as ti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09221_gb300 import build
    build.build()
    import paper_2604_09221_gb300 as e
    e.library()
    return e


def regular(eng, d, lo, hi, flags=0):
    tri = eng.Triangulation(d, ti.regular_triangulation(d, seed=40 + d))
    h = eng.Histogram(4096, tri.code_words)
    eng.enumerate_schemes(tri, lo, hi, h, flags)
    codes, counts, failed = h.read()
    assert failed == 0
    return tri, collections.Counter(dict(zip(codes[:, 0].tolist(), counts.tolist())))


def no_alloc_raw(eng, tri, lo, hi, flags=0, cap=2048):
    """One call through the C ABI; returns (codes, counts, [n, failed, err])."""
    import torch
    codes = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    counts = torch.zeros(max(cap, 1), dtype=torch.int64, device="cuda")
    n_out = torch.zeros(3, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = eng.library().ts_enumerate_noalloc(tri.handle, lo, hi, flags, codes.data_ptr(),
                                            counts.data_ptr(), cap, n_out.data_ptr(), stream)
    assert st == 0
    torch.cuda.synchronize()
    return (codes.cpu().numpy().view(np.uint64), counts.cpu().numpy().view(np.uint64),
            [int(x) for x in n_out.cpu().tolist()])


def no_alloc(eng, tri, lo, hi, flags=0, cap=2048):
    codes, counts, (n, failed, err) = no_alloc_raw(eng, tri, lo, hi, flags, cap)
    assert failed == 0 and err == 0 and n <= cap
    return collections.Counter(dict(zip(codes[:n].tolist(), counts[:n].tolist())))


@pytest.mark.parametrize("d,lo,hi,flags", [(6, 1000, 1000 + (1 << 20), 0), (7, 12345, 12345 + 300001, 0),
                                           (5, 0, 1 << 18, 2), (9, 777, 777 + (1 << 16), 1)])
def test_no_alloc_matches_ts_enumerate_twice(eng, d, lo, hi, flags):
    tri, want = regular(eng, d, lo, hi, flags)
    assert no_alloc(eng, tri, lo, hi, flags) == want
    assert no_alloc(eng, tri, lo, hi, flags) == want   # second call on the reused array


def test_no_alloc_rejects_oversized_capacity(eng):
    import torch
    tri = eng.Triangulation(4, ti.standard_triangulation(4))
    buf = torch.zeros(4096, dtype=torch.int64, device="cuda")
    st = eng.library().ts_enumerate_noalloc(tri.handle, 0, 16, 0, buf.data_ptr(), buf.data_ptr(),
                                            4096, buf.data_ptr(), None)
    assert st == 1  # TS_EINVAL: more than the 2048 codes the static table holds


def test_no_alloc_overflow_keeps_count_and_sets_flag(eng):
    """More distinct codes than cap: n_out[0] is still the true number of
    codes, only cap (code, count) pairs are written, each one of the sweep's,
    and the overflow bit (2) is set in n_out[2]."""
    lo, hi = 1000, 1000 + (1 << 20)
    tri, want = regular(eng, 6, lo, hi)
    assert len(want) > 2
    codes, counts, (n, failed, err) = no_alloc_raw(eng, tri, lo, hi, 0, cap=2)
    assert n == len(want) and failed == 0 and err & 2
    for c, k in zip(codes[:2].tolist(), counts[:2].tolist()):
        assert want[c] == k
    # the next call, within its capacity, is clean again
    assert no_alloc(eng, tri, lo, hi) == want
