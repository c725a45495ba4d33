"""GPU: mixed-degree batches (one graph launch of per-degree persistent
kernels).  Every job's histogram equals the oracle's on the same splitmix64
sign vectors, the per-instance codes too; a job gives the same result alone
and in the mix, with and without the graph, on replay, and after a tile
change; the autotuner returns tiles that run."""
import collections

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


def job_base(seed, stream):
    # the counter base that tcurve_inputs.random_masks uses for one-word masks
    return ti.splitmix64_int(((seed & ((1 << 64) - 1)) * 0x100000001B3 + stream) & ((1 << 64) - 1))


@pytest.fixture(scope="module")
def jobs(eng):
    rng = np.random.default_rng(5)
    out = []
    for d in (4, 5, 6, 7, 8, 9):
        for k, e in enumerate(ti.regular_triangulations(d, 2, seed=300 + d)):
            n = int(rng.integers(1000, 30000))
            out.append((d, e, n, 1000 + d, k))
    return out


def oracle_hist(orc, d, e, n, seed, stream):
    masks = ti.random_masks(n, d, seed, stream)
    codes = orc.real_schemes(d, orc.triangles(d, e), masks)
    return codes[:, 0], collections.Counter(codes[:, 0].tolist())


def hist_of(batch, j):
    codes, counts, failed = batch.read(j)
    assert failed == 0
    return collections.Counter(dict(zip(codes.tolist(), counts.tolist())))


def test_batch_matches_oracle_alone_and_in_the_mix(eng, orc, jobs):
    import torch
    tris = [eng.Triangulation(d, e) for d, e, *_ in jobs]
    counts = [n for _, _, n, _, _ in jobs]
    bases = [job_base(s, k) for *_, s, k in jobs]
    outs = [torch.zeros(n, dtype=torch.int64, device="cuda") if i % 3 == 0 else None
            for i, n in enumerate(counts)]
    batch = eng.Batch(tris, counts, bases, code_outputs=outs)
    batch.run(graph=True)
    got = [hist_of(batch, j) for j in range(len(jobs))]
    for j, (d, e, n, s, k) in enumerate(jobs):
        codes, want = oracle_hist(orc, d, e, n, s, k)
        assert got[j] == want, (j, d)
        if outs[j] is not None:
            assert (outs[j].cpu().numpy().view(np.uint64) == codes).all()
    # replay, no graph, a tile change: same results
    batch.run(graph=True)
    assert [hist_of(batch, j) for j in range(len(jobs))] == got
    batch.run(graph=False)
    assert [hist_of(batch, j) for j in range(len(jobs))] == got
    batch.set_tile(7, 64, 64 * 4)
    batch.run(graph=True)
    assert [hist_of(batch, j) for j in range(len(jobs))] == got
    batch.set_tile(8, 128, 128 * 4, eng.TS_SCRATCH_GLOBAL)   # scratch in global memory
    batch.set_tile(6, 96, 96 * 16, eng.TS_SCRATCH_SHARED)
    batch.run(graph=True)
    assert [hist_of(batch, j) for j in range(len(jobs))] == got
    # each job alone
    for j in (0, 5, len(jobs) - 1):
        alone = eng.Batch([tris[j]], [counts[j]], [bases[j]])
        alone.run()
        assert hist_of(alone, 0) == got[j]


def test_autotuner_picks_tiles_that_run(eng, jobs, tmp_path):
    from paper_2604_09221_gb300 import autotune
    sel = [x for x in jobs if x[0] in (6, 9)]
    tris = [eng.Triangulation(d, e) for d, e, *_ in sel]
    counts = [n for _, _, n, _, _ in sel]
    bases = [job_base(s, k) for *_, s, k in sel]
    cache = str(tmp_path / "tiles.json")
    tiles = autotune.autotune(tris, counts, bases, cache=cache, reps=1,
                              threads=(64, 128), chunk_per_thread=(4, 16))
    assert set(tiles) == {6, 9}
    again = autotune.autotune(tris, counts, bases, cache=cache, reps=1)
    assert again == tiles  # served from the cache
    batch = eng.Batch(tris, counts, bases)
    autotune.apply(batch, tiles)
    batch.run()
    for j in range(len(sel)):
        assert sum(hist_of(batch, j).values()) == counts[j]


def test_mixed_batch_full_size(eng, orc):
    """The mixed-degree batch workload at its full size: 32 seeded regular
    triangulations for each d in 5..10, 2^U(10,24) splitmix64 sign vectors
    per triangulation (about 3.3e8 in all), one graph launch, the groups of
    d = 5 and 6 on specialised code and the others table-driven.  Every job's
    histogram accounts for all its sign vectors, none failed, and every
    scheme satisfies the classical restrictions; one job per degree also
    stores its codes, and 1024 sampled rows of each equal the oracle's codes
    of the same sign vectors."""
    import torch
    from schemes import check_classical
    degrees, per_degree, seed = (5, 6, 7, 8, 9, 10), 32, 31
    rng = np.random.default_rng(seed)
    tris, edges, counts, bases = [], [], [], []
    for d in degrees:
        for k, e in enumerate(ti.regular_triangulations(d, per_degree, seed=seed + d)):
            tris.append(eng.Triangulation(d, e))
            edges.append(e)
            counts.append(int(2 ** rng.uniform(10, 24)))
            bases.append(job_base(seed * 100 + d, k))
    sampled = [degrees.index(d) * per_degree for d in degrees]   # first job of each degree
    outs = [torch.zeros((counts[j], tris[j].code_words), dtype=torch.int64, device="cuda")
            if j in sampled else None for j in range(len(tris))]
    batch = eng.Batch(tris, counts, bases, code_outputs=outs)
    for d in degrees:   # specialised code up to d = 6 (every group is large enough)
        assert batch.info(d)["kernel"] == ("specialized" if d <= 6 else "table"), \
            batch.info(d)["log"][-2000:]
    batch.run(graph=True)
    torch.cuda.synchronize()
    checked = set()
    for j, t in enumerate(tris):
        codes, cnt, failed = batch.read(j)
        assert failed == 0 and int(cnt.sum()) == counts[j], j
        for c in codes.reshape(len(cnt), -1):
            key = (t.d, eng.code_to_int(c))
            if key not in checked:
                assert check_classical(*key) == [], key
                checked.add(key)
    for j in sampled:
        d, n = tris[j].d, counts[j]
        idx = np.unique(np.concatenate([rng.integers(0, n, 1024), [0, n - 1]]))
        signs = np.concatenate([ti.splitmix_sign_vectors(d, bases[j] + int(i), 1) for i in idx])
        want = orc.real_schemes(d, orc.triangles(d, edges[j]), signs)
        got = outs[j].cpu().numpy().view(np.uint64)[idx]
        assert (got == want).all(), (d, j)


def specialised_jobs(eng, degrees, seed, max_n):
    """Two triangulations per degree and three jobs per degree: the first
    triangulation twice (one ts_tri in two jobs), the second once."""
    rng = np.random.default_rng(seed)
    jobs = []
    for d in degrees:
        es = ti.regular_triangulations(d, 2, seed=seed + d)
        ts = [eng.Triangulation(d, e) for e in es]
        for k, i in enumerate((0, 1, 0)):
            jobs.append({"d": d, "edges": es[i], "tri": ts[i], "n": int(rng.integers(1, max_n)),
                         "base": job_base(seed * 10 + d, k)})
    return jobs


def test_specialised_batch_matches_oracle(eng, orc):
    """Specialised batch groups (each triangulation compiled into a
    straight-line sweep of its own, linked with the group's persistent
    kernel) for degrees 3..12: one and two sign and code words, narrow and
    wide back ends, ragged counts, codes stored for every other job.  Every
    job's histogram and stored codes equal the oracle's on the same
    splitmix64 sign vectors, in one graph launch, on replay, after a chunk
    change, and after a switch to the table-driven kernel and back; a tile
    of another block size is refused; the degree groups run one after the
    other give the same results as run concurrently."""
    import torch
    degrees = (3, 5, 6, 7, 8, 9, 10, 11, 12)
    jobs = specialised_jobs(eng, degrees, 700, 6000)
    tris = [j["tri"] for j in jobs]
    outs = [torch.zeros((j["n"], j["tri"].code_words), dtype=torch.int64, device="cuda")
            if i % 2 == 0 else None for i, j in enumerate(jobs)]
    batch = eng.Batch(tris, [j["n"] for j in jobs], [j["base"] for j in jobs], code_outputs=outs)
    for d in degrees:
        batch.set_kernel(d, eng.TS_KERNEL_SPECIALIZED)
        info = batch.info(d)
        assert info["kernel"] == "specialized" and info["threads"] == 128, info["log"][-2000:]
    batch.run(graph=True)
    got = []
    for i, j in enumerate(jobs):
        codes, cnt, failed = batch.read(i)
        assert failed == 0
        h = collections.Counter({eng.code_to_int(c): int(k)
                                 for c, k in zip(codes.reshape(len(cnt), -1), cnt)})
        want = orc.real_schemes(j["d"], orc.triangles(j["d"], j["edges"]),
                                ti.splitmix_sign_vectors(j["d"], j["base"], j["n"]))
        assert h == collections.Counter(orc.code_to_int(w) for w in want), (i, j["d"])
        if outs[i] is not None:
            assert (outs[i].cpu().numpy().view(np.uint64) == want).all(), (i, j["d"])
        got.append(h)

    def hists():
        out = []
        for i in range(len(jobs)):
            codes, cnt, failed = batch.read(i)
            assert failed == 0
            out.append(collections.Counter({eng.code_to_int(c): int(k)
                                            for c, k in zip(codes.reshape(len(cnt), -1), cnt)}))
        return out
    batch.run(graph=True)
    assert hists() == got
    batch.set_tile(10, 128, 128 * 2, eng.TS_SCRATCH_GLOBAL)
    batch.run(graph=True)
    assert hists() == got
    with pytest.raises(eng.TSError):
        batch.set_tile(10, 64, 64 * 16, eng.TS_SCRATCH_GLOBAL)
    batch.set_kernel(7, eng.TS_KERNEL_TABLE)
    assert batch.info(7)["kernel"] == "table"
    batch.run(graph=False)
    assert hists() == got
    batch.set_kernel(7, eng.TS_KERNEL_SPECIALIZED)
    batch.run(graph=True)
    assert hists() == got
    batch.set_serial(True)     # degree groups one after the other
    batch.run(graph=True)
    assert hists() == got
    batch.run(graph=False)
    assert hists() == got


def test_specialised_batch_by_size(eng):
    """TS_KERNEL_AUTO at creation: a degree group of d <= 6 with at least
    2^22 sign vectors runs specialised code; a smaller one, one of higher
    degree, and one with a triangulation set to TS_KERNEL_TABLE run the
    table-driven kernel; the large groups count all their sign vectors."""
    t5 = [eng.Triangulation(5, e) for e in ti.regular_triangulations(5, 2, seed=505)]
    t6 = eng.Triangulation(6, ti.regular_triangulation(6, seed=606))
    t8 = eng.Triangulation(8, ti.regular_triangulation(8, seed=808))
    t9 = eng.Triangulation(9, ti.regular_triangulation(9, seed=909))
    t9.set_kernel(eng.TS_KERNEL_TABLE)
    counts = [1 << 21, 1 << 21, 5000, 1 << 23, 1 << 22]
    batch = eng.Batch(t5 + [t6, t8, t9], counts, [1, 2, 3, 4, 5])
    assert batch.info(5)["kernel"] == "specialized", batch.info(5)["log"][-2000:]
    assert batch.info(6)["kernel"] == "table"
    assert batch.info(8)["kernel"] == "table"
    assert batch.info(9)["kernel"] == "table"
    batch.run()
    for j, n in enumerate(counts):
        codes, cnt, failed = batch.read(j)
        assert failed == 0 and int(cnt.sum()) == n
