"""GPU parity of the warp-per-instance kernels (TS_KERNEL_WARP): one warp
classifies one sign vector, lanes sharing a lock-free union-find in shared
memory.  Codes and enumeration histograms through the C ABI against the CPU
oracle on the same seeded inputs, bit for bit, at every degree (one and
several sign and code words), on standard, regular and fan triangulations,
with ragged batch sizes, special sign vectors, every mask map, and a sampled
check of a full-size sweep against the table-driven kernel."""
import collections

import numpy as np
import pytest

import tcurve_inputs as ti

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


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


def warp_tri(eng, d, edges):
    tri = eng.Triangulation(d, edges)
    tri.set_kernel(eng.TS_KERNEL_WARP)
    return tri


def gpu_codes(tri, masks):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(masks).view(np.int64)).cuda()
    return tri.real_schemes(t).cpu().numpy().view(np.uint64)


def words_of(d, values):
    W = ti.sign_words(d)
    return np.array([[(v >> (64 * w)) & M64 for w in range(W)] for v in values], dtype=np.uint64)


def hist_rows(hist):
    codes, counts, failed = hist.read()
    assert failed == 0
    return collections.Counter({tuple(int(x) for x in c): int(k) for c, k in zip(codes, counts)})


def counter(codes):
    return collections.Counter(tuple(int(x) for x in row) for row in codes)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_exhaustive_small_degrees(eng, orc, d):
    masks = np.arange(1 << ti.num_points(d), dtype=np.uint64).reshape(-1, 1)
    cases = [ti.standard_triangulation(d)]
    if d >= 3:
        cases.append(ti.regular_triangulation(d, seed=500 + d))
    if d >= 2:
        cases.append(ti.fan_triangulation(d))
    for e in cases:
        got = gpu_codes(warp_tri(eng, d, e), masks)
        assert (got == orc.real_schemes(d, orc.triangles(d, e), masks)).all(), d


@pytest.mark.parametrize("d", list(range(5, 17)))
def test_random_sign_vectors(eng, orc, d):
    """Standard, regular and fan triangulations; a batch that spans several
    blocks and ends in a ragged tail."""
    n = 20011 if d <= 12 else 4099
    for idx, e in enumerate([ti.standard_triangulation(d), ti.regular_triangulation(d, seed=510 + d),
                             ti.fan_triangulation(d)]):
        masks = ti.random_masks(n, d, 900 + d, stream=idx)
        got = gpu_codes(warp_tri(eng, d, e), masks)
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert bad.size == 0, (d, idx, bad[:5])


@pytest.mark.parametrize("d", [6, 9, 10, 16])
def test_special_sign_vectors(eng, orc, d):
    """Constant signs, Harnack's distribution and the parity patterns (the
    M-curves and one-region schemes), and stray bits above |A|."""
    A = ti.num_points(d)
    vals = [0, (1 << A) - 1]
    for rule in (lambda i, j: i % 2 == 0 and j % 2 == 0, lambda i, j: i % 2 == 1 and j % 2 == 1,
                 lambda i, j: (i + j) % 2 == 0, lambda i, j: i % 2 == 0,
                 lambda i, j: (i % 2 == 0) != (j % 2 == 0)):
        v = 0
        for j in range(d + 1):
            for i in range(d + 1 - j):
                if rule(i, j):
                    v |= 1 << (j * (d + 1) - j * (j - 1) // 2 + i)
        vals.append(v)
    e = ti.regular_triangulation(d, seed=520 + d)
    masks = words_of(d, vals)
    want = orc.real_schemes(d, orc.triangles(d, e), masks)
    tri = warp_tri(eng, d, e)
    assert (gpu_codes(tri, masks) == want).all()
    W = ti.sign_words(d)
    top = A - 64 * (W - 1)   # sign bits in the last word
    if top < 64:
        stray = masks.copy()
        stray[:, W - 1] |= np.uint64(M64 ^ ((1 << top) - 1))
        assert (gpu_codes(tri, stray) == want).all()


@pytest.mark.parametrize("n", [0, 1, 7, 31, 32, 33, 255, 257])
def test_batch_sizes(eng, orc, n):
    d = 11
    e = ti.regular_triangulation(d, seed=530)
    masks = ti.random_masks(max(n, 1), d, 531, stream=n)[:n]
    tri = warp_tri(eng, d, e)
    if n == 0:
        import torch
        out = tri.real_schemes(torch.zeros((0, ti.sign_words(d)), dtype=torch.int64, device="cuda"))
        assert out.shape[0] == 0
        return
    assert (gpu_codes(tri, masks) == orc.real_schemes(d, orc.triangles(d, e), masks)).all()


def enum_values(d, flags, lo, hi, eng):
    out = []
    for k in range(lo, hi):
        if flags == eng.TS_ENUM_FLIP:
            out.append(k << 1)
        elif flags == eng.TS_ENUM_REDUCED:
            out.append(((k & ((1 << (d - 1)) - 1)) << 2) | ((k >> (d - 1)) << (d + 2)))
        else:
            out.append(k)
    return out


@pytest.mark.parametrize("d", [5, 8, 10, 13, 16])
def test_enumerate_against_oracle(eng, orc, d):
    """Every mask map over a ragged range (not a multiple of the 128
    instances a warp takes at once), block-private histograms (d <= 9) and
    direct multi-word inserts (d >= 10)."""
    e = ti.regular_triangulation(d, seed=540 + d)
    tri = warp_tri(eng, d, e)
    otri = orc.triangles(d, e)
    h = eng.Histogram(8192, tri.code_words)
    lo = (1 << 40) + 12345 if d >= 7 else 123
    n = 6007 if d <= 11 else 2003
    for flags in (0, eng.TS_ENUM_FLIP, eng.TS_ENUM_REDUCED, eng.TS_ENUM_SPLITMIX):
        if flags != eng.TS_ENUM_SPLITMIX and d < 7:
            continue
        h.clear()
        eng.enumerate_schemes(tri, lo, lo + n, h, flags)
        if flags == eng.TS_ENUM_SPLITMIX:
            masks = ti.splitmix_sign_vectors(d, lo, n)
        else:
            masks = words_of(d, enum_values(d, flags, lo, lo + n, eng))
        assert hist_rows(h) == counter(orc.real_schemes(d, otri, masks)), (d, flags)


def test_enumerate_full_range_d5(eng, orc):
    d = 5
    e = ti.fan_triangulation(d)
    tri = warp_tri(eng, d, e)
    n = 1 << ti.num_points(d)
    h = eng.Histogram(4096, tri.code_words)
    eng.enumerate_schemes(tri, 0, n, h)
    masks = np.arange(n, dtype=np.uint64).reshape(-1, 1)
    assert hist_rows(h) == counter(orc.real_schemes(d, orc.triangles(d, e), masks))


@pytest.mark.parametrize("d", [10, 16])
def test_sweep_agrees_with_table_kernel(eng, d):
    """A larger splitmix64 sweep: the warp kernel's histogram equals the
    table-driven kernel's (which the wide tests check against the oracle)."""
    e = ti.regular_triangulation(d, seed=d)
    n = 1 << 20 if d == 10 else 1 << 18
    rows = []
    for kind in (eng.TS_KERNEL_WARP, eng.TS_KERNEL_TABLE):
        tri = eng.Triangulation(d, e)
        tri.set_kernel(kind)
        h = eng.Histogram(1 << 21, tri.code_words)   # room for every instance's own scheme
        eng.enumerate_schemes(tri, 0, n, h, eng.TS_ENUM_SPLITMIX)
        rows.append(hist_rows(h))
    assert sum(rows[0].values()) == n
    assert rows[0] == rows[1]
