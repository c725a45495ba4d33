"""Input generators (tcurve_inputs): the splitmix64 finaliser against the
published outputs of the generator, the layout of multi-word sign vectors,
and the lattice sizes of the seeded triangulations.  CPU only."""
import numpy as np
import pytest

import tcurve_inputs as ti

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def test_splitmix64_matches_the_published_sequence():
    # splitmix64 seeded with 0 (Steele, Lea, Flood): state += GOLDEN, output
    # = finaliser(state); its first three outputs
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [ti.splitmix64_int((GOLDEN * i) & M64) for i in range(3)]
    assert got == want
    arr = ti.splitmix64(np.array([(GOLDEN * i) & M64 for i in range(3)], dtype=np.uint64))
    assert [int(x) for x in arr] == want


@pytest.mark.parametrize("d", [1, 7, 9, 10, 13, 16])
def test_splitmix_sign_vectors_layout(d):
    base, n = (1 << 63) + 12345, 50
    W, npts = ti.sign_words(d), ti.num_points(d)
    v = ti.splitmix_sign_vectors(d, base, n)
    assert v.shape == (n, W) and v.dtype == np.uint64
    for i in (0, 1, n - 1):
        k = (base + i) & M64
        for w in range(W):
            x = ti.splitmix64_int((k * W + w) & M64)
            if w == W - 1 and npts - 64 * w < 64:
                x &= (1 << (npts - 64 * w)) - 1
            assert int(v[i, w]) == x
    # no bit at or above |A|
    top = npts - 64 * (W - 1)
    if top < 64:
        assert not (v[:, -1] >> np.uint64(top)).any()


@pytest.mark.parametrize("d", [1, 7, 10, 16])
def test_random_masks_clear_high_bits(d):
    m = ti.random_masks(500, d, seed=3)
    top = ti.num_points(d) - 64 * (ti.sign_words(d) - 1)
    assert m.shape == (500, ti.sign_words(d))
    if top < 64:
        assert not (m[:, -1] >> np.uint64(top)).any()


@pytest.mark.parametrize("d", [3, 6, 10])
def test_regular_triangulations_are_unimodular_and_distinct(d):
    tris = ti.regular_triangulations(d, 4, seed=11)
    keys = set()
    for e in tris:
        # |E(T)| = 3d(d+1)/2 for a unimodular triangulation of d*Delta_2 (Euler)
        assert len(e) == 3 * d * (d + 1) // 2
        pts = {(int(r[0]), int(r[1])) for r in e} | {(int(r[2]), int(r[3])) for r in e}
        assert len(pts) == ti.num_points(d)       # every lattice point is a vertex
        keys.add(tuple(sorted(tuple(sorted(((int(r[0]), int(r[1])), (int(r[2]), int(r[3]))))) for r in e)))
    assert len(keys) == len(tris)
