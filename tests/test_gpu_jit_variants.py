"""GPU parity of the specialised kernels in every configuration: shared or
global per-thread scratch, and the register budgets of several resident
blocks per SM.  Codes (query kernel) and sweep histograms (per-mask and
block sweeps, every mask map) must equal the oracle's."""
import collections

import numpy as np
import pytest

import tcurve_inputs as ti

pytestmark = pytest.mark.gpu
CONFIGS = [(2, 0), (2, 4), (2, 6), (2, 8), (1, 3)]  # (TS_SCRATCH_*, blocks per SM)


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


def enum_masks(d, flags, lo, hi, eng):
    k = np.arange(lo, hi, dtype=np.uint64)
    if flags == eng.TS_ENUM_FLIP:
        return (k << np.uint64(1)).reshape(-1, 1)
    if flags == eng.TS_ENUM_REDUCED:
        low = k & np.uint64((1 << (d - 1)) - 1)
        return ((low << np.uint64(2)) | ((k >> np.uint64(d - 1)) << np.uint64(d + 2))).reshape(-1, 1)
    return k.reshape(-1, 1)


@pytest.mark.parametrize("where,blocks", CONFIGS)
@pytest.mark.parametrize("d", [5, 7, 9])
def test_specialised_configurations(eng, orc, d, where, blocks):
    import torch
    e = ti.regular_triangulation(d, seed=600 + d)
    otri = orc.triangles(d, e)
    tri = eng.Triangulation(d, e)
    tri.set_kernel(eng.TS_KERNEL_SPECIALIZED)
    tri.set_scratch(where)
    tri.set_occupancy(blocks)
    tri.prepare()
    masks = ti.random_masks(9001, d, 7, stream=where * 16 + blocks)
    got = tri.real_schemes(torch.from_numpy(masks.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    assert (got == orc.real_schemes(d, otri, masks)).all()
    h = eng.Histogram(4096, 1)
    # a ragged range that spans several whole middle-row blocks (block sweep)
    width = 1 << (d + 3)
    for flags in (0, eng.TS_ENUM_FLIP, eng.TS_ENUM_REDUCED):
        lo = 12345 if flags != eng.TS_ENUM_REDUCED else 999
        h.clear()
        eng.enumerate_schemes(tri, lo, lo + width, h, flags)
        codes, counts, failed = h.read()
        assert failed == 0
        want = collections.Counter(orc.real_schemes(d, otri, enum_masks(d, flags, lo, lo + width, eng))[:, 0].tolist())
        assert dict(zip(codes[:, 0].tolist(), counts.tolist())) == dict(want), (d, flags)
