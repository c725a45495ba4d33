"""GPU: a checkpointed sweep through ts_enumerate (stopped and resumed) gives
the histogram of one uninterrupted sweep, which equals the oracle's on a
sub-range; sharding a range into parts and merging gives the same histogram."""
import collections

import numpy as np
import pytest

import tcurve_inputs as ti
from paper_2604_09221_gb300 import sweep

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


def test_checkpointed_engine_sweep(eng, orc, tmp_path):
    d = 7
    edges = ti.regular_triangulation(d, seed=123)
    tri = eng.Triangulation(d, edges)
    fn = sweep.engine_chunk_fn(tri)
    lo, hi, chunk = 3, 3 + (1 << 26) + 1000, 1 << 23
    path = str(tmp_path / "d7.json")
    a = sweep.CheckpointedSweep(lo, hi, chunk, path, fn, tag="d7")
    a.run(max_chunks=2)
    b = sweep.CheckpointedSweep(lo, hi, chunk, path, fn, tag="d7")
    got = b.run()
    assert b.done and got == fn(lo, hi) and sum(got.values()) == hi - lo
    parts = [sweep.shard_range(lo, hi, r, 5) for r in range(5)]
    assert sweep.merge(*(fn(x, y) for x, y in parts)) == got
    ks = np.arange(lo, lo + 40000, dtype=np.uint64).reshape(-1, 1)
    want = collections.Counter(orc.real_schemes(d, orc.triangles(d, edges), ks)[:, 0].tolist())
    assert fn(lo, lo + 40000) == dict(want)
