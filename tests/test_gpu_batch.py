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
