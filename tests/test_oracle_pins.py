"""Pins of the CPU oracle to facts fixed by the paper and by classical
mathematics (not to the oracle itself).

* hand enumerations: d = 1 (Harnack bound M = 1, one pseudoline), d = 2 (all
  four unimodular triangulations of 2*Delta_2; a conic has one oval), a hand
  trace of d = 2 with sigma = 0, d = 3 (J or J + <1>);
* the classification of quartics (5 nonempty schemes) and quintics (8);
* Harnack's construction: the Harnack sign distribution on the anti-diagonal
  triangulation gives Harnack's M-curve scheme;
* Harnack, Petrovskii, Gudkov-Rokhlin, Kharlamov-Gudkov-Krakhnov, Bezout;
* the GF(2)-rank Betti numbers of the curve and of its complement (the
  "mod 2 homology" method named in Sec. 2) on small degrees;
* symmetry: the (Z/2)^3 action on signs and the S_3 action (Sec. 3);
* Fig. 2: the printed oval-count distributions of three degree-8
  triangulations, on a uniform sample, and the bow tie's restriction to even
  oval counts stated beside the figure.
"""
import collections
import itertools
import math
import os

import numpy as np
import pytest

import tcurve_inputs as ti
from schemes import (check_classical, code_of, harnack_M, ovals, parity_counts,
                     rohlin_viro, tree_of)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lat(d, i, j):
    return j * (d + 1) - j * (j - 1) // 2 + i


def points(d):
    return [(i, j) for j in range(d + 1) for i in range(d + 1 - j)]


def all_masks(d):
    return np.arange(1 << ti.num_points(d), dtype=np.uint64).reshape(-1, 1)


def load_edges(name):
    return np.loadtxt(os.path.join(GOLDEN, f"fig2_{name}.edges"), dtype=np.int32, comments="#")


# ---------------------------------------------------------------------------
# code format worked values
# ---------------------------------------------------------------------------

def test_code_format_worked_values():
    assert code_of([]) == 1
    assert code_of([[]]) == 6
    assert code_of([[], []]) == 26
    assert code_of([[]] * 3) == 106
    assert code_of([[]] * 4) == 426
    assert code_of([[[]]]) == 28
    assert code_of([[[]], [], []]) == 458
    assert rohlin_viro(6, 458) == "<1<1> + 2>"
    assert rohlin_viro(7, 6) == "<J + 1>"
    for c in (1, 6, 26, 28, 106, 426, 458):
        assert code_of(tree_of(c)) == c


# ---------------------------------------------------------------------------
# hand enumerations
# ---------------------------------------------------------------------------

def test_d1_every_curve_is_a_pseudoline(orc):
    tri = orc.triangles(1, ti.standard_triangulation(1))
    codes, st = orc.real_schemes(1, tri, all_masks(1), with_stats=True)
    assert set(codes[:, 0].tolist()) == {1}
    assert (st[:, 1] == 1).all() and (st[:, 0] == 0).all()


D2_TRIANGULATIONS = {
    # the four unimodular triangulations of 2*Delta_2 (two S_3 orbits)
    "standard": [((0, 0), (1, 0), (0, 1)), ((1, 0), (2, 0), (1, 1)),
                 ((0, 1), (1, 1), (0, 2)), ((1, 0), (1, 1), (0, 1))],
    "fan00": [((0, 0), (1, 0), (1, 1)), ((1, 0), (2, 0), (1, 1)),
              ((0, 0), (1, 1), (0, 1)), ((0, 1), (1, 1), (0, 2))],
    "fan20": [((2, 0), (0, 1), (1, 0)), ((0, 0), (1, 0), (0, 1)),
              ((2, 0), (1, 1), (0, 1)), ((0, 1), (1, 1), (0, 2))],
    "fan02": [((0, 2), (1, 0), (0, 1)), ((0, 0), (1, 0), (0, 1)),
              ((0, 2), (1, 0), (1, 1)), ((1, 0), (2, 0), (1, 1))],
}


def edges_of(tris):
    es = set()
    for t in tris:
        for a in range(3):
            p, q = sorted((t[a], t[(a + 1) % 3]))
            es.add((p, q))
    return np.array([[p[0], p[1], q[0], q[1]] for p, q in sorted(es)], dtype=np.int32)


@pytest.mark.parametrize("name", sorted(D2_TRIANGULATIONS))
def test_d2_every_curve_is_one_oval(orc, name):
    tri = orc.triangles(2, edges_of(D2_TRIANGULATIONS[name]))
    codes, st = orc.real_schemes(2, tri, all_masks(2), with_stats=True)
    assert set(codes[:, 0].tolist()) == {6}
    assert (st[:, 0] == 1).all() and (st[:, 1] == 0).all()


def test_d2_hand_trace_sigma_zero(orc):
    # sigma = 0 on the standard triangulation: by Eq. 2 the negative diamond
    # points are (0,-1), (1,-1), (-1,0), (-1,1).  Counting by hand: 14 edges
    # of T^diamond join a negative and a positive point, 12 of the 16
    # triangles are mixed, 4 crossed boundary edges form 2 antipodal pairs,
    # so the curve has 14 - 2 = 12 vertices and 12 segments: one cycle.
    tri = orc.triangles(2, ti.standard_triangulation(2))
    code, st = orc.real_scheme(2, tri, 0)
    assert code == 6
    assert st["n_crossed"] == 14 and st["n_segments"] == 12
    assert st["n_ovals"] == 1 and st["n_pseudolines"] == 0


def test_d3_schemes(orc):
    seen = set()
    tris = [ti.standard_triangulation(3)] + ti.regular_triangulations(3, 3, seed=3)
    for e in tris:
        tri = orc.triangles(3, e)
        codes, st = orc.real_schemes(3, tri, all_masks(3), with_stats=True)
        assert set(codes[:, 0].tolist()) <= {1, 6}
        assert (st[:, 1] == 1).all()
        seen |= set(codes[:, 0].tolist())
    assert seen == {1, 6}


QUARTICS = {code_of(t) for t in ([[]], [[], []], [[]] * 3, [[]] * 4, [[[]]])}
QUINTICS = {code_of([[]] * k) for k in range(7)} | {code_of([[[]]])}


def test_d4_exhaustive_quartic_schemes(orc):
    seen = set()
    for e in [ti.standard_triangulation(4)] + ti.regular_triangulations(4, 3, seed=4):
        tri = orc.triangles(4, e)
        codes = orc.real_schemes(4, tri, all_masks(4))[:, 0]
        assert set(codes.tolist()) <= QUARTICS
        seen |= set(codes.tolist())
    assert seen == QUARTICS


def test_d5_quintic_schemes(orc):
    seen = set()
    for e in [ti.standard_triangulation(5)] + ti.regular_triangulations(5, 2, seed=5):
        tri = orc.triangles(5, e)
        codes = orc.real_schemes(5, tri, ti.random_masks(1 << 14, 5, 5))[:, 0]
        assert set(codes.tolist()) <= QUINTICS
        seen |= set(codes.tolist())
    assert len(seen) >= 7


# ---------------------------------------------------------------------------
# Harnack's M-curves
# ---------------------------------------------------------------------------

def harnack_sigma(d):
    s = 0
    for (i, j) in points(d):
        if i % 2 == 0 and j % 2 == 0:
            s |= 1 << lat(d, i, j)
    return s


@pytest.mark.parametrize("d", [4, 6, 8, 10, 12])
def test_harnack_distribution_even_degree(orc, d):
    # Harnack's M-curve of degree 2k: <3k(k-1)/2 + 1<(k-1)(k-2)/2>>
    k = d // 2
    tri = orc.triangles(d, ti.standard_triangulation(d))
    code, st = orc.real_scheme(d, tri, harnack_sigma(d))
    assert code == code_of([[]] * (3 * k * (k - 1) // 2) + [[[]] * ((k - 1) * (k - 2) // 2)])
    assert st["n_ovals"] == harnack_M(d)


def test_harnack_distribution_quintic(orc):
    tri = orc.triangles(5, ti.standard_triangulation(5))
    code, st = orc.real_scheme(5, tri, harnack_sigma(5))
    assert code == code_of([[]] * 6) and st["n_pseudolines"] == 1


# ---------------------------------------------------------------------------
# classical restrictions on regular triangulations
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,n", [(6, 1 << 14), (7, 1 << 13), (8, 1 << 12)])
def test_classical_restrictions(orc, d, n):
    seen = set()
    for idx, e in enumerate([ti.standard_triangulation(d)] + ti.regular_triangulations(d, 4, seed=d)):
        tri = orc.triangles(d, e)
        sig = ti.random_masks(n, d, 100 + d, stream=idx)
        codes, st = orc.real_schemes(d, tri, sig, with_stats=True)
        assert (st[:, 1] == d % 2).all()
        assert (st[:, 0] + st[:, 1] <= harnack_M(d)).all()
        for c in set(codes[:, 0].tolist()):
            assert check_classical(d, c) == [], (d, c, rohlin_viro(d, c))
        for c, row in zip(codes[:64, 0].tolist(), st[:64]):
            t = tree_of(c)
            assert ovals(t) == row[0]
            p, nn = parity_counts(t)
            assert (p, nn) == (row[3], row[4])
        seen |= set(codes[:, 0].tolist())
    # all nonempty real schemes of degree 6 number 55, of degree 7 number 121
    assert len(seen) <= {6: 55, 7: 121}.get(d, 10**9)


# ---------------------------------------------------------------------------
# GF(2) Betti numbers of the curve and of its complement
# ---------------------------------------------------------------------------

def gf2_rank(rows):
    """Rank over GF(2) of a list of int bitsets."""
    rank = 0
    piv = {}
    for r in rows:
        while r:
            h = r.bit_length() - 1
            if h in piv:
                r ^= piv[h]
            else:
                piv[h] = r
                rank += 1
                break
    return rank


def diamond_cells(d, tri, sigma):
    """Cells of S (Sec. 2) built here independently: vertex classes, edge
    classes and triangles of T^diamond with antipodal boundary identification,
    and the vertex signs of Eq. 2."""
    def sgn(x, y):
        i, j = abs(x), abs(y)
        s = (sigma >> lat(d, i, j)) & 1
        if x < 0:
            s ^= i & 1
        if y < 0:
            s ^= j & 1
        return s

    def on_bd(p):
        return abs(p[0]) + abs(p[1]) == d

    def vcls(p):
        if on_bd(p):
            q = (-p[0], -p[1])
            return min(p, q)
        return p

    tris = []
    for (sx, sy) in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        for t in tri:
            tris.append(tuple((sx * int(t[2 * k]), sy * int(t[2 * k + 1])) for k in range(3)))
    edges = {}
    for t in tris:
        for a in range(3):
            p, q = sorted((t[a], t[(a + 1) % 3]))
            edges.setdefault((p, q), []).append(t)

    def ecls(e):
        p, q = e
        if on_bd(p) and on_bd(q):
            f = tuple(sorted(((-p[0], -p[1]), (-q[0], -q[1]))))
            return min(e, f)
        return e

    return sgn, vcls, ecls, tris, edges


def betti0_curve_and_complement(d, tri, sigma):
    sgn, vcls, ecls, tris, edges = diamond_cells(d, tri, sigma)
    crossed = {e for e in edges if sgn(*e[0]) != sgn(*e[1])}
    # curve: 0-cells = crossed edge classes, 1-cells = mixed triangles
    c0 = sorted({ecls(e) for e in crossed})
    idx0 = {c: n for n, c in enumerate(c0)}
    rows = []
    for t in tris:
        es = [tuple(sorted((t[a], t[(a + 1) % 3]))) for a in range(3)]
        cr = [e for e in es if e in crossed]
        if cr:
            assert len(cr) == 2
            rows.append((1 << idx0[ecls(cr[0])]) ^ (1 << idx0[ecls(cr[1])]))
    b0_curve = len(c0) - gf2_rank(rows)
    # complement: vertex classes joined by classes of non-crossed edges
    vs = sorted({vcls(p) for e in edges for p in e})
    iv = {v: n for n, v in enumerate(vs)}
    rows = []
    for e in {ecls(e) for e in edges if e not in crossed}:
        rows.append((1 << iv[vcls(e[0])]) ^ (1 << iv[vcls(e[1])]))
    b0_regions = len(vs) - gf2_rank(rows)
    n_cells = (len(vs), len({ecls(e) for e in edges}), len(tris))
    return b0_curve, b0_regions, n_cells


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_gf2_betti_numbers(orc, d):
    for idx, e in enumerate([ti.standard_triangulation(d)] + ti.regular_triangulations(d, 2, seed=40 + d)):
        tri = orc.triangles(d, e)
        sig = ti.random_masks(48, d, 7 * d, stream=idx)
        codes, st = orc.real_schemes(d, tri, sig, with_stats=True)
        for s, row in zip(sig[:, 0].tolist(), st):
            b_curve, b_reg, (nv, ne, nf) = betti0_curve_and_complement(d, tri, int(s))
            assert nv - ne + nf == 1  # Euler characteristic of RP^2
            assert b_curve == row[0] + row[1]
            assert b_reg == row[0] + 1


# ---------------------------------------------------------------------------
# symmetry (Sec. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [4, 5, 6, 7])
def test_sign_symmetry_z2_cubed(orc, d):
    tri = orc.triangles(d, ti.regular_triangulations(d, 1, seed=90 + d)[0])
    full = (1 << ti.num_points(d)) - 1
    imask = sum(1 << lat(d, i, j) for (i, j) in points(d) if i % 2)
    jmask = sum(1 << lat(d, i, j) for (i, j) in points(d) if j % 2)
    sig = ti.random_masks(512, d, 3, stream=d)
    base = orc.real_schemes(d, tri, sig)[:, 0]
    for g in (full, imask, jmask, imask ^ jmask ^ full):
        other = orc.real_schemes(d, tri, sig ^ np.uint64(g))[:, 0]
        assert (other == base).all()


@pytest.mark.parametrize("d", [4, 6, 7])
def test_coordinate_permutation_symmetry(orc, d):
    e = ti.regular_triangulations(d, 1, seed=70 + d)[0]
    tri = orc.triangles(d, e)
    sig = ti.random_masks(256, d, 11, stream=d)
    base = orc.real_schemes(d, tri, sig)[:, 0]
    perms = [lambda i, j: (j, i), lambda i, j: (d - i - j, j), lambda i, j: (i, d - i - j)]
    for pi in perms:
        e2 = np.array([[*pi(a, b), *pi(c, dd)] for a, b, c, dd in e], dtype=np.int32)
        tri2 = orc.triangles(d, e2)
        sig2 = np.zeros_like(sig)
        for (i, j) in points(d):
            i2, j2 = pi(i, j)
            bit = (sig >> np.uint64(lat(d, i, j))) & np.uint64(1)
            sig2 |= bit << np.uint64(lat(d, i2, j2))
        assert (orc.real_schemes(d, tri2, sig2)[:, 0] == base).all()


# ---------------------------------------------------------------------------
# Fig. 2: three degree-8 triangulations and their oval-count distributions
# ---------------------------------------------------------------------------

def fig2_percentages():
    out = collections.defaultdict(dict)
    with open(os.path.join(GOLDEN, "fig2_oval_percentages.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            name, k, p = line.split()
            out[name][int(k)] = float(p)
    return out


@pytest.mark.parametrize("name", ["bow_tie", "rank016", "rank015"])
def test_fig2_triangulation_data(orc, name):
    e = load_edges(name)
    assert len(e) == 3 * 8 * 9 // 2
    tri = orc.triangles(8, e)
    assert len(tri) == 64
    if name == "rank016":
        sw = {tuple(sorted([(a, b), (c, dd)])) for a, b, c, dd in e}
        assert sw == {tuple(sorted([(b, a), (dd, c)])) for a, b, c, dd in e}


@pytest.mark.parametrize("name", ["bow_tie", "rank016", "rank015"])
def test_fig2_oval_count_distribution(orc, name):
    N = 1 << 17
    tri = orc.triangles(8, load_edges(name))
    codes, st = orc.real_schemes(8, tri, ti.random_masks(N, 8, 2026, stream={"bow_tie": 1, "rank016": 2, "rank015": 3}[name]),
                                 with_stats=True)
    counts = collections.Counter(st[:, 0].tolist())
    printed = fig2_percentages()[name]
    assert abs(sum(printed.values()) - 100.0) < 0.01
    for k in range(23):
        p = printed.get(k, 0.0) / 100.0
        q = counts.get(k, 0) / N
        sd = math.sqrt(max(p * (1 - p), 1.0 / N) / N)
        assert abs(q - p) <= 5 * sd + 1e-6, (name, k, p, q)
    if name == "bow_tie":
        assert all(k % 2 == 0 for k in counts)
