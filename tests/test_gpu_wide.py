"""GPU parity for the multi-word degrees 10..16 (|A| = 66..153: two or three
sign words, two to four code words, up to 107 regions): query codes,
enumeration histograms under every mask map, the device splitmix64 stream,
mixed-degree batches and the server, all against the CPU oracle on the same
seeded inputs, bit for bit."""
import collections

import numpy as np
import pytest

import tcurve_inputs as ti

pytestmark = pytest.mark.gpu
WIDE = [10, 11, 12, 13, 14, 15, 16]
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


def gpu_codes(tri, masks):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(masks).view(np.int64)).cuda()
    return tri.real_schemes(t).cpu().numpy().view(np.uint64)


def words_of(d, values):
    """(n, W) uint64 sign words of Python-int sign vectors."""
    W = ti.sign_words(d)
    return np.array([[(v >> (64 * w)) & M64 for w in range(W)] for v in values], dtype=np.uint64)


def counter(codes):
    return collections.Counter(tuple(int(x) for x in row) for row in codes)


def hist_rows(hist):
    codes, counts, failed = hist.read()
    assert failed == 0
    return collections.Counter({tuple(int(x) for x in c): int(k) for c, k in zip(codes, counts)})


@pytest.mark.parametrize("d", WIDE)
def test_random_sign_vectors_wide(eng, orc, d):
    """Random sign vectors of the standard, a regular and the fan
    triangulation (its origin has 4d - 1 earlier neighbours) against the
    oracle."""
    n = 20011 if d <= 12 else 4099   # several blocks and a ragged tail
    for idx, e in enumerate([ti.standard_triangulation(d), ti.regular_triangulation(d, seed=40 + d),
                             ti.fan_triangulation(d)]):
        tri = eng.Triangulation(d, e)
        assert (tri.sign_words, tri.code_words) == (ti.sign_words(d), orc.code_words(d))
        masks = ti.random_masks(n, d, 61 + d, stream=idx)
        got = gpu_codes(tri, masks)
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert bad.size == 0, (d, idx, bad[:5])


@pytest.mark.parametrize("d,where", [(5, 2), (7, 1), (7, 2), (9, 1), (9, 2), (10, 1), (13, 1), (16, 1), (16, 2)])
def test_scratch_placements(eng, orc, d, where):
    """Shared- and global-memory scratch give the oracle's codes and sweep
    histograms (TS_SCRATCH_SHARED = 1, TS_SCRATCH_GLOBAL = 2)."""
    e = ti.regular_triangulation(d, seed=500 + d)
    tri = eng.Triangulation(d, e)
    tri.set_kernel(eng.TS_KERNEL_TABLE)
    tri.set_scratch(where)
    otri = orc.triangles(d, e)
    masks = ti.random_masks(3001, d, 5, stream=where)
    assert (gpu_codes(tri, masks) == orc.real_schemes(d, otri, masks)).all()
    h = eng.Histogram(8192, tri.code_words)
    eng.enumerate_schemes(tri, 77, 77 + 2500, h, eng.TS_ENUM_SPLITMIX)
    assert hist_rows(h) == counter(orc.real_schemes(d, otri, ti.splitmix_sign_vectors(d, 77, 2500)))


@pytest.mark.parametrize("d", WIDE)
def test_special_sign_vectors_wide(eng, orc, d):
    pts = [(i, j) for j in range(d + 1) for i in range(d + 1 - j)]
    full = (1 << len(pts)) - 1
    harnack = sum(1 << n for n, (i, j) in enumerate(pts) if i % 2 == 0 and j % 2 == 0)
    odd = sum(1 << n for n, (i, j) in enumerate(pts) if i % 2 == 1 and j % 2 == 1)
    alt = sum(1 << n for n, (i, j) in enumerate(pts) if (i + j) % 2)
    masks = words_of(d, [0, full, harnack, odd, alt, full ^ alt, 1, full >> 1, 1 << 64, (1 << 64) - 1])
    for e in (ti.standard_triangulation(d), ti.regular_triangulation(d, seed=d)):
        tri = eng.Triangulation(d, e)
        got = gpu_codes(tri, masks)
        assert (got == orc.real_schemes(d, orc.triangles(d, e), masks)).all()
    # Harnack's distribution on the anti-diagonal triangulation is an M-curve
    # (M = (d-1)(d-2)/2 + 1 components: ovals, plus the pseudoline for odd d)
    tri = eng.Triangulation(d, ti.standard_triangulation(d))
    code = gpu_codes(tri, masks[2:3])[0]
    nbits = max(64 * w + int(code[w]).bit_length() - 1 for w in range(len(code)) if code[w])
    M = (d - 1) * (d - 2) // 2 + 1
    assert nbits // 2 == (M if d % 2 == 0 else M - 1)


@pytest.mark.parametrize("d", [10, 16])
def test_stray_high_bits_wide(eng, d):
    tri = eng.Triangulation(d, ti.regular_triangulation(d, seed=3))
    masks = ti.random_masks(2048, d, 4)
    dirty = masks.copy()
    top = ti.num_points(d) - 64 * (ti.sign_words(d) - 1)
    dirty[:, -1] |= np.uint64(0x5A5A5A5A5A5A5A5A) << np.uint64(top) if top < 64 else np.uint64(0)
    assert (gpu_codes(tri, masks) == gpu_codes(tri, dirty)).all()


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1025])
def test_batch_sizes_wide(eng, orc, n):
    import torch
    d = 12
    e = ti.regular_triangulation(d, seed=12)
    tri = eng.Triangulation(d, e)
    masks = ti.random_masks(max(n, 1), d, 9)[:n]
    got = tri.real_schemes(torch.from_numpy(masks.view(np.int64)).cuda().reshape(-1, tri.sign_words))
    assert got.shape == (n, tri.code_words)
    if n:
        want = orc.real_schemes(d, orc.triangles(d, e), masks)
        assert (got.cpu().numpy().view(np.uint64) == want).all()
    host = tri.real_schemes_host(masks) if n else None
    if n:
        assert (host == want).all()


@pytest.mark.parametrize("d", [4, 10, 13, 16])
def test_device_splitmix_stream(eng, d):
    base = (0xC0FFEE << 40) | d
    got = eng.splitmix_masks(d, base, 1000).cpu().numpy().view(np.uint64).reshape(1000, -1)
    assert (got == ti.splitmix_sign_vectors(d, base, 1000)).all()


def enum_values(d, flags, lo, hi, eng):
    """Python-int sign vectors of the mask maps of ts_enumerate."""
    out = []
    for k in range(lo, hi):
        if flags == eng.TS_ENUM_FLIP:
            out.append(k << 1)
        elif flags == eng.TS_ENUM_REDUCED:
            out.append(((k & ((1 << (d - 1)) - 1)) << 2) | ((k >> (d - 1)) << (d + 2)))
        else:
            out.append(k)
    return out


@pytest.mark.parametrize("d", [10, 11, 14, 16])
def test_enumerate_wide_against_oracle(eng, orc, d):
    e = ti.regular_triangulation(d, seed=70 + d)
    tri = eng.Triangulation(d, e)
    otri = orc.triangles(d, e)
    h = eng.Histogram(8192, tri.code_words)
    lo = (1 << 62) + 12345
    n = 6007 if d <= 11 else 2003
    for flags in (0, eng.TS_ENUM_FLIP, eng.TS_ENUM_REDUCED, eng.TS_ENUM_SPLITMIX):
        h.clear()
        eng.enumerate_schemes(tri, lo, lo + n, h, flags)
        if flags == eng.TS_ENUM_SPLITMIX:
            masks = ti.splitmix_sign_vectors(d, lo, n)
        else:
            masks = words_of(d, enum_values(d, flags, lo, lo + n, eng))
        want = counter(orc.real_schemes(d, otri, masks))
        assert hist_rows(h) == want, (d, flags)


def test_wide_batch_and_mix(eng, orc):
    """A batch holding degrees 5, 10, 12 and 16: histograms and codes equal the
    oracle's on the jobs' splitmix64 streams."""
    import torch
    rng = np.random.default_rng(17)
    spec = [(5, 3000), (10, 5000), (10, 700), (12, 2500), (16, 1200), (16, 33)]
    edges = [ti.regular_triangulation(d, seed=900 + i) for i, (d, _) in enumerate(spec)]
    tris = [eng.Triangulation(d, e) for (d, _), e in zip(spec, edges)]
    counts = [n for _, n in spec]
    bases = [int(rng.integers(0, 1 << 62)) for _ in spec]
    outs = [torch.zeros((n, t.code_words), dtype=torch.int64, device="cuda") for (_, n), t in zip(spec, tris)]
    batch = eng.Batch(tris, counts, bases, code_outputs=outs)
    for graph in (True, False):
        batch.run(graph=graph)
        for j, ((d, n), e) in enumerate(zip(spec, edges)):
            codes, cnt, failed = batch.read(j)
            assert failed == 0
            rows = codes.reshape(len(cnt), -1)
            got = collections.Counter({tuple(int(x) for x in c): int(k) for c, k in zip(rows, cnt)})
            want_codes = orc.real_schemes(d, orc.triangles(d, e), ti.splitmix_sign_vectors(d, bases[j], n))
            assert got == counter(want_codes), (j, d)
            assert (outs[j].cpu().numpy().view(np.uint64) == want_codes).all(), (j, d)
    batch.close()


def test_server_with_wide_jobs(eng, orc):
    """Jobs of degrees 6 and 10..16 on the server: each equals the oracle on
    its splitmix64 stream, run concurrently with the others."""
    from paper_2604_09221_gb300.serve import GpuExecutor, Job, Server
    degrees = [6, 10, 12, 14, 16]
    edges = [(d, ti.regular_triangulation(d, seed=800 + d)) for d in degrees]
    tris = [eng.Triangulation(d, e) for d, e in edges]
    rng = np.random.default_rng(23)
    jobs = [dict(tri=i % len(tris), n=int(rng.integers(200, 1500)), base=int(rng.integers(0, 1 << 62)),
                 want_codes=(i % 2 == 0)) for i in range(15)]
    srv = Server(GpuExecutor(tris, slots=4, kernel=eng.TS_KERNEL_TABLE), slots=4, mem_budget=1 << 30)
    got = [f.result(timeout=600) for f in [srv.submit(Job(**j)) for j in jobs]]
    srv.close()
    for j, g in zip(jobs, got):
        d, e = edges[j["tri"]]
        want = orc.real_schemes(d, orc.triangles(d, e), ti.splitmix_sign_vectors(d, j["base"], j["n"]))
        wh = collections.Counter(int(sum(int(x) << (64 * w) for w, x in enumerate(r))) for r in want)
        assert g.hist == dict(wh), (d, j["n"])
        if j["want_codes"]:
            assert (np.asarray(g.codes).reshape(want.shape) == want).all()


def test_bounded_wait_reports_a_timeout(eng):
    """A device wait that nothing completes gives up after its limit and
    reports TS_ETIMEOUT; the context stays usable afterwards."""
    import torch
    assert eng.selftest_wait(2048) == 6   # TS_ETIMEOUT
    tri = eng.Triangulation(6, ti.regular_triangulation(6, seed=1))
    x = torch.zeros(64, dtype=torch.int64, device="cuda")
    assert tri.real_schemes(x).shape == (64, 1)


def test_histogram_overflow_is_reported(eng):
    """A histogram with room for far fewer codes than the sweep produces
    reports TS_EOVERFLOW (bounded probing, error word) instead of losing
    counts silently."""
    tri = eng.Triangulation(12, ti.regular_triangulation(12, seed=12))
    h = eng.Histogram(2, tri.code_words)       # 16 slots
    eng.enumerate_schemes(tri, 0, 20000, h, eng.TS_ENUM_SPLITMIX)
    with pytest.raises(eng.TSError) as ex:
        h.read()
    assert ex.value.status == 5
