"""GPU: the bench's workload whole against the oracle.  ts_enumerate over
masks [0, 2^32) of tcurve_inputs.regular_triangulation(7, seed=7), in the
launch configuration bench.py times (the triangulation's specialised block
sweep, default tile), gives exactly the histogram that the CPU oracle gives
for the same 2^32 masks, bin by bin.  The expected histogram is stored in
tests/golden/d7_seed7_sweep_2p32.hist, written by
tests/golden/make_d7_sweep_histogram.py from oracle/ alone."""
import os

import numpy as np
import pytest

import tcurve_inputs as ti

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "d7_seed7_sweep_2p32.hist")


def load_golden():
    edges, hist, rng = None, {}, None
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("# edge "):
                edges = [tuple(int(x) for x in e.split(",")) for e in line[7:].split()]
            elif line.startswith("# range "):
                rng = tuple(int(x) for x in line.split()[2:4])
            elif not line.startswith("#") and line.strip():
                c, n = line.split()
                hist[int(c)] = int(n)
    return edges, rng, hist


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


def test_golden_file_is_the_benchs_triangulation_and_range():
    edges, rng, hist = load_golden()
    want = sorted(tuple(int(x) for x in r) for r in np.asarray(ti.regular_triangulation(7, seed=7)).reshape(-1, 4))
    assert edges == want and rng == (0, 1 << 32) and sum(hist.values()) == 1 << 32
    assert len(hist) <= 121   # at most the 121 real schemes of degree 7


def test_golden_histogram_holds_the_oracles_first_masks(orc):
    """A spot check of the stored file against the oracle itself: every
    scheme of the first 2^12 masks is a key of the stored histogram."""
    edges, _, hist = load_golden()
    d = 7
    codes = orc.real_schemes(d, orc.triangles(d, np.asarray(edges)),
                             np.arange(1 << 12, dtype=np.uint64).reshape(-1, 1))
    assert set(codes[:, 0].tolist()) <= set(hist)


@pytest.mark.gpu
def test_bench_sweep_equals_the_oracle_histogram(eng):
    edges, (lo, hi), want = load_golden()
    tri = eng.Triangulation(7, np.asarray(edges, dtype=np.int32))
    tri.prepare()
    h = eng.Histogram(4096, tri.code_words)
    eng.enumerate_schemes(tri, lo, hi, h)
    codes, counts, failed = h.read()
    assert failed == 0
    assert dict(zip(codes[:, 0].tolist(), counts.tolist())) == want
