"""GPU: the continuous-batching server.  Jobs of mixed degree and size run
concurrently (several slots, overlapping streams); each job's histogram and
codes equal those of the same job run alone, and small jobs equal the oracle."""
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


def test_results_alone_equal_results_in_the_mix(eng, orc):
    from paper_2604_09221_gb300.serve import GpuExecutor, Job, Server
    edges = [(d, ti.regular_triangulation(d, seed=500 + 10 * d + k)) for d in (6, 7, 8, 9) for k in range(2)]
    tris = [eng.Triangulation(d, e) for d, e in edges]
    rng = np.random.default_rng(11)
    jobs = []
    for i in range(48):
        t = int(rng.integers(0, len(tris)))
        n = int(2 ** rng.uniform(8, 16))
        jobs.append(dict(tri=t, n=n, base=int(rng.integers(0, 1 << 62)), want_codes=(i % 4 == 0)))
    mixed = Server(GpuExecutor(tris, slots=6, kernel=eng.TS_KERNEL_TABLE), slots=6, mem_budget=1 << 30)
    futs = [mixed.submit(Job(**j)) for j in jobs]
    got = [f.result(timeout=300) for f in futs]
    mixed.close()
    assert mixed.peak_running > 1
    alone = Server(GpuExecutor(tris, slots=1, kernel=eng.TS_KERNEL_TABLE), slots=1, mem_budget=1 << 30)
    for j, g in zip(jobs, got):
        r = alone.submit(Job(**j)).result(timeout=300)
        assert r.hist == g.hist
        assert sum(g.hist.values()) == j["n"]
        if j["want_codes"]:
            assert (r.codes == g.codes).all()
            assert collections.Counter(g.codes.tolist()) == g.hist
    alone.close()
    # small jobs against the oracle (same splitmix64 stream)
    for j, g in list(zip(jobs, got))[:6]:
        d, e = edges[j["tri"]]
        masks = np.array([ti.splitmix64_int((j["base"] + i) & ((1 << 64) - 1)) & ((1 << ti.num_points(d)) - 1)
                          for i in range(j["n"])], dtype=np.uint64).reshape(-1, 1)
        want = collections.Counter(orc.real_schemes(d, orc.triangles(d, e), masks)[:, 0].tolist())
        assert g.hist == dict(want)
