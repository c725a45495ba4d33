"""GPU: the fused batch launch (ts_batch_set_fused), one persistent kernel
for every job of every degree.  Each job's histogram and stored codes equal
the oracle's on the same splitmix64 sign vectors in every register tier
(largest degree 6, 9, 11, 16), with thread and warp tiles, chunk changes,
graph replay and launches without a graph, and the same as the per-degree
group launches of the same batch; malformed tiles are refused; jobs that
bring their own sign vectors run beside jobs on their streams."""
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


def make_jobs(eng, spec, seed):
    """spec: (degree, sign vectors) per job; the second job of a degree
    reuses the first one's ts_tri (one triangulation in two jobs)."""
    rng = np.random.default_rng(seed)
    jobs, first = [], {}
    for i, (d, n) in enumerate(spec):
        if d in first:
            e, t = first[d]
        else:
            e = ti.regular_triangulation(d, seed=seed + 10 * i)
            t = eng.Triangulation(d, e)
            first[d] = (e, t)
        jobs.append({"d": d, "n": n, "edges": e, "tri": t, "base": int(rng.integers(0, 1 << 62))})
    return jobs


def oracle_codes(orc, j):
    d = j["d"]
    return orc.real_schemes(d, orc.triangles(d, j["edges"]), ti.splitmix_sign_vectors(d, j["base"], j["n"]))


def hists(eng, batch, njobs):
    out = []
    for i in range(njobs):
        codes, cnt, failed = batch.read(i)
        assert failed == 0
        out.append(collections.Counter({eng.code_to_int(c): int(k)
                                        for c, k in zip(codes.reshape(len(cnt), -1), cnt)}))
    return out


TIERS = {
    6: [(3, 2000), (5, 3000), (5, 129), (6, 4100)],
    9: [(4, 1000), (7, 5000), (8, 300), (8, 2600), (9, 3000)],
    11: [(5, 1500), (9, 1000), (10, 2048), (10, 77), (11, 1500)],
    16: [(6, 1000), (9, 700), (12, 900), (13, 600), (16, 700), (16, 1)],
}


@pytest.mark.parametrize("tier", sorted(TIERS))
def test_fused_launch_matches_oracle(eng, orc, tier):
    import torch
    jobs = make_jobs(eng, TIERS[tier], 4000 + tier)
    tris = [j["tri"] for j in jobs]
    outs = [torch.zeros((j["n"], j["tri"].code_words), dtype=torch.int64, device="cuda")
            if i % 2 == 0 else None for i, j in enumerate(jobs)]
    batch = eng.Batch(tris, [j["n"] for j in jobs], [j["base"] for j in jobs], code_outputs=outs)
    batch.set_fused(True)
    for d in {j["d"] for j in jobs}:
        info = batch.info(d)
        assert info["kernel"] == "table" and info["threads"] == 128 and info["chunk"] == 1024
        assert info["local_bytes"] <= 256, info   # a few spilled words at most
    want = []
    for i, j in enumerate(jobs):
        w = oracle_codes(orc, j)
        want.append(collections.Counter(orc.code_to_int(c) for c in w))
        j["want_codes"] = w
    batch.run(graph=True)
    assert hists(eng, batch, len(jobs)) == want
    for i, j in enumerate(jobs):
        if outs[i] is not None:
            assert (outs[i].cpu().numpy().view(np.uint64) == j["want_codes"]).all(), (i, j["d"])
    batch.run(graph=True)                       # replay
    assert hists(eng, batch, len(jobs)) == want
    batch.set_fused_tile(max(TIERS[tier])[0], eng.TS_KERNEL_TABLE, 128 * 3)   # ragged work items
    batch.run(graph=False)
    assert hists(eng, batch, len(jobs)) == want
    if tier >= 9:                               # warp tiles run in the widest tier's kernel
        for d in {j["d"] for j in jobs if j["d"] >= 7}:
            batch.set_fused_tile(d, eng.TS_KERNEL_WARP, 256)
            assert batch.info(d)["kernel"] == "warp"
        batch.run(graph=True)
        assert hists(eng, batch, len(jobs)) == want
        for i, j in enumerate(jobs):
            if outs[i] is not None:
                assert (outs[i].cpu().numpy().view(np.uint64) == j["want_codes"]).all(), (i, j["d"])
    batch.set_fused(False)                      # the per-degree group launches: same results
    batch.run(graph=True)
    assert hists(eng, batch, len(jobs)) == want
    batch.close()


def test_fused_tiles_are_validated(eng):
    jobs = make_jobs(eng, [(5, 500), (8, 500)], 4100)
    batch = eng.Batch([j["tri"] for j in jobs], [j["n"] for j in jobs], [j["base"] for j in jobs])
    for args in ((5, eng.TS_KERNEL_WARP, 1024),      # no warp bodies below d = 7
                 (8, eng.TS_KERNEL_TABLE, 100),      # not a multiple of 128
                 (8, eng.TS_KERNEL_TABLE, 0),
                 (8, eng.TS_KERNEL_SPECIALIZED, 1024),
                 (9, eng.TS_KERNEL_TABLE, 1024)):    # no job of degree 9
        with pytest.raises(eng.TSError):
            batch.set_fused_tile(*args)
    batch.set_fused_tile(8, eng.TS_KERNEL_WARP, 512)  # set before the fused mode: kept
    batch.set_fused(True)
    assert batch.info(8)["kernel"] == "warp" and batch.info(8)["chunk"] == 512
    batch.run()
    for i, j in enumerate(jobs):
        codes, cnt, failed = batch.read(i)
        assert failed == 0 and int(cnt.sum()) == j["n"]
    batch.close()


def test_fused_launch_with_caller_sign_vectors(eng, orc):
    """Jobs that classify the caller's sign vectors (ts_batch_set_signs)
    beside jobs on their splitmix64 streams, in one fused launch, with thread
    and warp tiles: codes and histograms equal the oracle's on the same
    vectors (one, two and three sign words); the per-degree group mode
    refuses to run such a batch; a job returned to its stream gives the
    stream's schemes again."""
    import torch
    jobs = make_jobs(eng, [(6, 3000), (6, 1000), (9, 2000), (11, 900), (16, 400)], 4200)
    tris = [j["tri"] for j in jobs]
    outs = [torch.zeros((j["n"], j["tri"].code_words), dtype=torch.int64, device="cuda") for j in jobs]
    batch = eng.Batch(tris, [j["n"] for j in jobs], [j["base"] for j in jobs], code_outputs=outs)
    given = {}
    for i in (0, 2, 3, 4):   # caller vectors; job 1 stays on its stream
        j = jobs[i]
        words = ti.random_masks(j["n"], j["d"], seed=4300 + i)
        given[i] = words
        batch.set_signs(i, torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda())
    with pytest.raises(eng.TSError):
        batch.run()                               # group mode: refused
    batch.set_fused(True)

    def check():
        got = hists(eng, batch, len(jobs))
        for i, j in enumerate(jobs):
            d = j["d"]
            if i in given:
                want = orc.real_schemes(d, orc.triangles(d, j["edges"]), given[i])
            else:
                want = oracle_codes(orc, j)
            assert got[i] == collections.Counter(orc.code_to_int(c) for c in want), (i, d)
            assert (outs[i].cpu().numpy().view(np.uint64) == want).all(), (i, d)
    batch.run(graph=True)
    check()
    batch.set_fused_tile(9, eng.TS_KERNEL_WARP, 256)   # warp tiles read the caller's vectors too
    batch.set_fused_tile(16, eng.TS_KERNEL_WARP, 512)
    batch.run(graph=False)
    check()
    batch.set_signs(3, None)                      # back to its splitmix64 stream
    del given[3]
    batch.run(graph=True)
    check()
    batch.close()
