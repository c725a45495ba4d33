"""GPU parity: codes from the CUDA path (through the C ABI) must equal the CPU
oracle's bit for bit on the same seeded inputs.

Covers every supported degree, seeded regular triangulations, the paper's
three degree-8 triangulations (Fig. 2), exhaustive small degrees, ragged
batch sizes, stray high bits, the host-buffer entry point, and the
enumeration kernel (all three mask maps) against oracle histograms,
including a full-size degree-7 sweep checked on a sampled sub-range and by
properties that hold at any size.
"""
import collections
import os

import numpy as np
import pytest

import tcurve_inputs as ti
from schemes import check_classical, orbit_mask

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


KINDS = ["table", "specialized"]


def load(eng, d, edges, kind):
    tri = eng.Triangulation(d, edges)
    if kind == "specialized":
        tri.set_kernel(eng.TS_KERNEL_SPECIALIZED)
        tri.prepare()
    else:
        tri.set_kernel(eng.TS_KERNEL_TABLE)
    return tri


def gpu_codes(eng, tri, masks):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(masks).view(np.int64)).cuda()
    return tri.real_schemes(t).cpu().numpy().view(np.uint64)


def triangulations(d, k=2, seed=0):
    out = [("standard", ti.standard_triangulation(d))]
    if d >= 3:
        out += [(f"regular{n}", e) for n, e in enumerate(ti.regular_triangulations(d, k, seed=1000 + d + seed))]
    return out


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_exhaustive_small_degrees(eng, orc, d, kind):
    masks = np.arange(1 << ti.num_points(d), dtype=np.uint64).reshape(-1, 1)
    for name, e in triangulations(d, 3 if kind == "table" else 1):
        tri = load(eng, d, e, kind)
        got = gpu_codes(eng, tri, masks)
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        assert (got == want).all(), (d, name)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [5, 6, 7, 8, 9])
def test_random_sign_vectors(eng, orc, d, kind):
    n = 20011  # several blocks and a ragged tail
    for idx, (name, e) in enumerate(triangulations(d, 3 if kind == "table" else 1)):
        masks = ti.random_masks(n, d, 31 + d, stream=idx)
        tri = load(eng, d, e, kind)
        got = gpu_codes(eng, tri, masks)
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert bad.size == 0, (d, name, bad[:5], masks[bad[:5]])


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [8, 9])
def test_fan_triangulation(eng, orc, d, kind):
    """A triangulation whose origin has 4d - 1 earlier neighbours in
    T^diamond (a fan far longer than a regular triangulation's), random sign
    vectors and a sweep of a range, both kernel families, against the
    oracle."""
    e = ti.fan_triangulation(d)
    masks = ti.random_masks(20011, d, 77, stream=d)
    tri = load(eng, d, e, kind)
    got = gpu_codes(eng, tri, masks)
    want = orc.real_schemes(d, orc.triangles(d, e), masks)
    assert (got == want).all()
    h = eng.Histogram(4096, tri.code_words)
    lo = 123456
    eng.enumerate_schemes(tri, lo, lo + 5000, h)
    codes, counts, failed = h.read()
    assert failed == 0
    ref = orc.real_schemes(d, orc.triangles(d, e), np.arange(lo, lo + 5000, dtype=np.uint64).reshape(-1, 1))
    assert dict(zip(codes[:, 0].tolist(), counts.tolist())) == dict(collections.Counter(ref[:, 0].tolist()))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name", ["bow_tie", "rank016", "rank015"])
def test_fig2_triangulations(eng, orc, name, kind):
    e = np.loadtxt(os.path.join(GOLDEN, f"fig2_{name}.edges"), dtype=np.int32, comments="#")
    masks = ti.random_masks(30000, 8, 99, stream=len(name))
    tri = load(eng, 8, e, kind)
    got = gpu_codes(eng, tri, masks)
    want = orc.real_schemes(8, orc.triangles(8, e), masks)
    assert (got == want).all()


@pytest.mark.parametrize("kind", KINDS)
def test_special_sign_vectors(eng, orc, kind):
    for d in range(1, 10):
        npts = ti.num_points(d)
        full = (1 << npts) - 1
        pts = [(i, j) for j in range(d + 1) for i in range(d + 1 - j)]
        harnack = sum(1 << n for n, (i, j) in enumerate(pts) if i % 2 == 0 and j % 2 == 0)
        alt = sum(1 << n for n, (i, j) in enumerate(pts) if (i + j) % 2)
        masks = np.array([[0], [full], [harnack], [alt], [full ^ alt], [1], [full >> 1]], dtype=np.uint64)
        for name, e in triangulations(d, 1)[: (2 if kind == "table" else 1)]:
            tri = load(eng, d, e, kind)
            assert (gpu_codes(eng, tri, masks) == orc.real_schemes(d, orc.triangles(d, e), masks)).all()


@pytest.mark.parametrize("kind", KINDS)
def test_stray_high_bits_are_ignored(eng, kind):
    d = 6
    e = ti.regular_triangulation(d, seed=5)
    tri = load(eng, d, e, kind)
    masks = ti.random_masks(4096, d, 1)
    dirty = masks | (np.uint64(0xABCDEF) << np.uint64(ti.num_points(d)))
    assert (gpu_codes(eng, tri, masks) == gpu_codes(eng, tri, dirty)).all()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [0, 1, 31, 127, 128, 129, 4097, 300001])
def test_batch_sizes(eng, orc, n, kind):
    import torch
    d = 7
    e = ti.regular_triangulation(d, seed=77)
    tri = load(eng, d, e, kind)
    masks = ti.random_masks(max(n, 1), d, 3)[:n]
    got = tri.real_schemes(torch.from_numpy(masks.view(np.int64)).cuda().reshape(-1, 1))
    assert got.shape == (n, 1)
    if n:
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        assert (got.cpu().numpy().view(np.uint64) == want).all()


def test_host_buffer_entry_point(eng, orc):
    d = 6
    e = ti.regular_triangulation(d, seed=8)
    tri = eng.Triangulation(d, e)
    masks = ti.random_masks(5000, d, 8)
    assert (tri.real_schemes_host(masks) == orc.real_schemes(d, orc.triangles(d, e), masks)).all()


def oracle_hist(orc, d, e, masks):
    codes = orc.real_schemes(d, orc.triangles(d, e), masks)
    return collections.Counter(codes[:, 0].tolist())


def gpu_hist(eng, tri, lo, hi, flags=0):
    """Histogram of ts_enumerate over [lo, hi)."""
    h = eng.Histogram(4096, tri.code_words)
    eng.enumerate_schemes(tri, lo, hi, h, flags)
    codes, counts, failed = h.read()
    assert failed == 0
    return collections.Counter(dict(zip(codes[:, 0].tolist(), counts.tolist())))


def reduced_masks(d, ks):
    ks = np.asarray(ks, dtype=np.uint64)
    low = ks & np.uint64((1 << (d - 1)) - 1)
    return ((low << np.uint64(2)) | ((ks >> np.uint64(d - 1)) << np.uint64(d + 2))).reshape(-1, 1)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [4, 5])
def test_enumerate_full_range(eng, orc, d, kind):
    e = ti.regular_triangulation(d, seed=50 + d)
    tri = load(eng, d, e, kind)
    n = 1 << ti.num_points(d)
    assert gpu_hist(eng, tri, 0, n) == oracle_hist(orc, d, e, np.arange(n, dtype=np.uint64).reshape(-1, 1))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [6, 7, 8, 9])
def test_enumerate_ragged_ranges_and_flags(eng, orc, d, kind):
    e = ti.regular_triangulation(d, seed=60 + d)
    tri = load(eng, d, e, kind)
    lo, hi = 123457, 123457 + 50001
    ks = np.arange(lo, hi, dtype=np.uint64)
    assert gpu_hist(eng, tri, lo, hi) == oracle_hist(orc, d, e, ks.reshape(-1, 1))
    assert gpu_hist(eng, tri, lo, hi, eng.TS_ENUM_FLIP) == oracle_hist(orc, d, e, (ks << np.uint64(1)).reshape(-1, 1))
    assert gpu_hist(eng, tri, lo, hi, eng.TS_ENUM_REDUCED) == oracle_hist(orc, d, e, reduced_masks(d, ks))


@pytest.mark.parametrize("kind", KINDS)
def test_enumerate_reduced_equals_full_over_8(eng, kind):
    # (Z/2)^3 acts freely and preserves schemes (Sec. 3): the full histogram is
    # 8 times the histogram over the representatives.
    d = 5
    e = ti.regular_triangulation(d, seed=3)
    tri = load(eng, d, e, kind)
    full = gpu_hist(eng, tri, 0, 1 << ti.num_points(d))
    red = gpu_hist(eng, tri, 0, 1 << (ti.num_points(d) - 3), eng.TS_ENUM_REDUCED)
    assert full == collections.Counter({k: 8 * v for k, v in red.items()})


@pytest.mark.parametrize("d", [5, 6])
def test_flip_sweep_pairs_complementary_blocks(eng, orc, d):
    """TS_ENUM_FLIP sweeps of the specialised kernel take a block of masks
    and the block of its complement together, as one block with every
    middle-row pattern (the global sign flip keeps the scheme).  Over the
    whole range, over ranges whose unpaired blocks lie below or above the
    paired ones (with ragged masks at both ends), against the oracle on
    the masks k << 1; and every class counted twice by the plain sweep."""
    e = ti.regular_triangulation(d, seed=80 + d)
    tri = load(eng, d, e, "specialized")
    N = ti.num_points(d)
    full = 1 << (N - 1)
    if d == 5:   # blocks of 2^5 values of k
        for lo, hi in ((0, full), (37 * 32 + 5, full - 99 * 32 - 9), (300 * 32 + 5, full - 99 * 32 - 9)):
            ks = np.arange(lo, hi, dtype=np.uint64)
            want = oracle_hist(orc, d, e, (ks << np.uint64(1)).reshape(-1, 1))
            assert gpu_hist(eng, tri, lo, hi, eng.TS_ENUM_FLIP) == want, (lo, hi)
    plain = gpu_hist(eng, tri, 0, 1 << N)
    flip = gpu_hist(eng, tri, 0, full, eng.TS_ENUM_FLIP)
    assert plain == collections.Counter({k: 2 * v for k, v in flip.items()})


@pytest.mark.parametrize("kind", KINDS + ["warp"])
def test_orbit_sweep(eng, orc, kind):
    """TS_ENUM_ORBITS: over the whole range the histogram of TS_ENUM_REDUCED
    (both pick one sign distribution per (Z/2)^3 class; d = 5, 6); over
    ranges with ragged ends around whole blocks the oracle's histogram of the
    same masks (d = 4, 7, 8, 9); refused for d = 1 and above d = 9."""
    def loadk(d, e):
        if kind != "warp":
            return load(eng, d, e, kind)
        t = eng.Triangulation(d, e)
        t.set_kernel(eng.TS_KERNEL_WARP)
        return t
    for d in (5, 6):
        e = ti.regular_triangulation(d, seed=90 + d)
        tri = loadk(d, e)
        full = 1 << (ti.num_points(d) - 3)
        assert gpu_hist(eng, tri, 0, full, eng.TS_ENUM_ORBITS) == \
            gpu_hist(eng, tri, 0, full, eng.TS_ENUM_REDUCED), d
    for d in ((4, 7) if kind == "warp" else (4, 7, 8, 9)):
        e = ti.regular_triangulation(d, seed=90 + d)
        tri = loadk(d, e)
        blk = 1 << (d + 1)
        lo = 3 * blk + 77
        hi = min(lo + 20 * blk + 999, 1 << (ti.num_points(d) - 3))
        masks = np.array([orbit_mask(d, k) for k in range(lo, hi)], dtype=np.uint64).reshape(-1, 1)
        assert gpu_hist(eng, tri, lo, hi, eng.TS_ENUM_ORBITS) == oracle_hist(orc, d, e, masks), d
    for d, status in ((1, 1), (10, 8)):   # TS_EINVAL, TS_EUNSUPPORTED
        t = eng.Triangulation(d, ti.standard_triangulation(d))
        h = eng.Histogram(64, t.code_words)
        with pytest.raises(eng.TSError) as err:
            eng.enumerate_schemes(t, 0, 64, h, eng.TS_ENUM_ORBITS)
        assert err.value.status == status


@pytest.mark.parametrize("kind", KINDS)
def test_enumerate_d7_full_size_slice(eng, orc, kind):
    """The benchmark workload (degree 7, masks [0, 2^32)) in the launch
    configuration the bench uses: every count accounted for, every scheme a
    valid septic scheme, no more than the 121 that exist, and the sub-range
    [2^31, 2^31 + 2^16) equal to the oracle's histogram."""
    d = 7
    e = ti.regular_triangulation(d, seed=7)
    tri = load(eng, d, e, kind)
    full = gpu_hist(eng, tri, 0, 1 << 32)
    assert sum(full.values()) == 1 << 32
    assert len(full) <= 121
    for c in full:
        assert check_classical(d, c) == []
    lo = 1 << 31
    ks = np.arange(lo, lo + (1 << 16), dtype=np.uint64).reshape(-1, 1)
    assert gpu_hist(eng, tri, lo, lo + (1 << 16)) == oracle_hist(orc, d, e, ks)


def test_kernels_agree_on_full_size_sweep(eng):
    """Table-driven and specialised sweeps of the bench slice give the same
    histogram (both are checked against the oracle on sub-ranges above)."""
    d = 7
    e = ti.regular_triangulation(d, seed=7)
    a = gpu_hist(eng, load(eng, d, e, "table"), 0, 1 << 32)
    b = gpu_hist(eng, load(eng, d, e, "specialized"), 0, 1 << 32)
    assert a == b


def test_d6_plain_full_size(eng, orc):
    """The degree-6 query workload at its full size: 64 distinct seeded
    regular triangulations, 2^20 uniform random sign vectors each (512 MiB of
    signs in all), through ts_real_schemes (table-driven kernel; the
    specialised kernel on four of them).  Per triangulation, 4096 sampled
    rows and the first and last rows equal the oracle's codes; at full size,
    no instance failed, every scheme satisfies the classical restrictions and
    at most 55 distinct nonempty sextic schemes occur."""
    d, n, k = 6, 1 << 20, 64
    tris = ti.regular_triangulations(d, k, seed=6)
    rng = np.random.default_rng(606)
    seen = set()
    for t, e in enumerate(tris):
        masks = ti.random_masks(n, d, seed=6, stream=t)
        tri = load(eng, d, e, "specialized" if t < 4 else "table")
        got = gpu_codes(eng, tri, masks)[:, 0]
        assert got.shape == (n,) and (got != 0).all()
        idx = np.unique(np.concatenate([rng.integers(0, n, 4096), [0, n - 1]]))
        want = orc.real_schemes(d, orc.triangles(d, e), masks[idx])[:, 0]
        assert (got[idx] == want).all(), t
        seen |= {int(c) for c in np.unique(got)}
    assert len(seen) <= 55
    for c in seen:
        assert check_classical(d, c) == [], c
