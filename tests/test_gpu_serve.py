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


def test_every_job_kind_alone_equals_the_mix(eng, orc):
    """Sample, query (host array and CUDA tensor) and enumeration jobs (no
    flag, TS_ENUM_FLIP, TS_ENUM_REDUCED) of degrees 6..9 and 11 on one server:
    each result equals the same job run alone; query codes equal the oracle's,
    enumeration histograms equal the oracle's over the same masks; an
    overflowing sample job is re-run with a histogram of its own."""
    import torch

    from paper_2604_09221_gb300.serve import GpuExecutor, Job, Server
    edges = [(d, ti.regular_triangulation(d, seed=900 + d)) for d in (6, 7, 8, 9, 11)]
    tris = [eng.Triangulation(d, e) for d, e in edges]
    rng = np.random.default_rng(17)

    def make(i):
        t = i % len(tris)
        d = edges[t][0]
        kind = ("sample", "query", "query_dev", "enum")[i % 4]
        n = int(2 ** rng.uniform(6, 13))
        if kind == "sample":
            return dict(tri=t, n=n, base=int(rng.integers(0, 1 << 62)), want_codes=bool(i % 8 == 0))
        if kind.startswith("query"):
            signs = ti.random_masks(n, d, 5000 + i)
            return dict(tri=t, kind="query", signs=signs, dev=kind == "query_dev")
        flags = (0, eng.TS_ENUM_FLIP, eng.TS_ENUM_REDUCED)[(i // 4) % 3]
        lo = int(rng.integers(0, 1 << 20))
        return dict(tri=t, kind="enum", lo=lo, hi=lo + n, flags=flags)

    specs = [make(i) for i in range(40)]

    def job(sp):
        sp = dict(sp)
        dev = sp.pop("dev", False)
        if sp.get("kind") == "query" and dev:
            sp["signs"] = torch.from_numpy(sp["signs"].view(np.int64)).cuda()
        return Job(**sp)

    def server(slots, classes=None):
        return Server(GpuExecutor(tris, slots=slots, kernel=eng.TS_KERNEL_TABLE, classes=classes),
                      slots=slots, mem_budget=1 << 32)

    mixed = server(6)
    got = [f.result(timeout=300) for f in [mixed.submit(job(s)) for s in specs]]
    mixed.close()
    assert mixed.peak_running > 1
    alone = server(1)
    for sp, g in zip(specs, got):
        r = alone.submit(job(sp)).result(timeout=300)
        assert r.hist == g.hist and r.kind == g.kind
        if g.codes is not None:
            assert (r.codes == g.codes).all()
    alone.close()
    for sp, g in zip(specs, got):
        d, e = edges[sp["tri"]]
        otri = orc.triangles(d, e)
        if sp.get("kind") == "query":
            want = orc.real_schemes(d, otri, sp["signs"])
            assert (g.codes.reshape(len(want), -1) == want).all()
            assert sum(g.hist.values()) == len(want)
        elif sp.get("kind") == "enum":
            ks = np.arange(sp["lo"], sp["hi"], dtype=np.uint64)
            if sp["flags"] == eng.TS_ENUM_FLIP:
                masks = ks << np.uint64(1)
            elif sp["flags"] == eng.TS_ENUM_REDUCED:
                low = ks & np.uint64((1 << (d - 1)) - 1)
                masks = (low << np.uint64(2)) | ((ks >> np.uint64(d - 1)) << np.uint64(d + 2))
            else:
                masks = ks
            words = np.zeros((len(masks), ti.sign_words(d)), dtype=np.uint64)
            words[:, 0] = masks   # the ranges here stay below bit 64
            want = orc.real_schemes(d, otri, words)
            assert g.hist == dict(collections.Counter(orc.code_to_int(w) for w in want))
        else:
            assert sum(g.hist.values()) == sp["n"]
    # a sample job with more schemes than the smallest resident class when
    # forced to it: re-run with its own histogram, same result as alone
    srv = server(2, classes=(16,))   # every job runs in the 16-code class first
    sp = dict(tri=4, n=4096, base=123)
    r = srv.submit(Job(**sp)).result(timeout=300)
    assert len(srv.requeued) == 1 and len(r.hist) > 16 and sum(r.hist.values()) == 4096
    srv.close()
