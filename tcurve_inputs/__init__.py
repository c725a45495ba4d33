"""Seeded synthetic inputs for T-curve workloads.

This module is shared by the CPU oracle side (``oracle/``, ``tests/``) and the
GPU side (``paper_2604_09221_gb300``, ``bench.py``).  It only *produces* inputs:
triangulations of d*Delta_2 given as edge lists of lattice points (Sec. 2
takes a triangulation as its list of edges) and bit-packed sign vectors.
It holds none of the method's arithmetic (no sign extension, no crossing test,
no component or nesting logic).

Generators
----------
* ``standard_triangulation(d)``: every unit square split by its anti-diagonal.
  It is the regular triangulation induced by the lifting i^2 + j^2 + (i+j)^2.
* ``regular_triangulation(d, seed, tri_id)``: the projection of the exact lower
  convex hull of the lifted points (i, j, omega(i, j)) (regularity, Sec. 2) with
  omega(i, j) = 1000 * (i^2 + j^2 + (i+j)^2) + U_int[0, 2000]; draws whose
  subdivision is not a unimodular triangulation (a point unused, a facet that
  is not a unit triangle, or a degenerate lifting) are rejected and redrawn.
* ``random_masks(...)``: counter-based splitmix64 sign words.
* ``splitmix_sign_vectors(d, base, n)``: the sign vectors of splitmix64
  counters base, base + 1, ...: word w of counter k is splitmix64(k * W + w),
  the top word cut to |A| bits (one word: splitmix64(k)).  The engine draws
  the same stream on the device (ts_splitmix_masks, TS_ENUM_SPLITMIX,
  batches and serving jobs).

Every value is reproducible from (seed, ids) alone.
"""
from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_int(x: int) -> int:
    """splitmix64 finaliser on one Python int (Steele, Lea, Flood 2014)."""
    z = (x + _GOLDEN) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 over a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(x, dtype=np.uint64) + np.uint64(_GOLDEN)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def num_points(d: int) -> int:
    """|A| = (d+1)(d+2)/2 (Eq. 1)."""
    return (d + 1) * (d + 2) // 2


def sign_words(d: int) -> int:
    return (num_points(d) + 63) // 64


# ----------------------------------------------------------------------------
# triangulations
# ----------------------------------------------------------------------------

def _edges_from_triangles(tris) -> np.ndarray:
    edges = set()
    for t in tris:
        for a in range(3):
            p, q = t[a], t[(a + 1) % 3]
            edges.add((p, q) if p < q else (q, p))
    out = np.array([[p[0], p[1], q[0], q[1]] for p, q in sorted(edges)], dtype=np.int32)
    return out.reshape(-1, 4)


def standard_triangulation(d: int) -> np.ndarray:
    """Anti-diagonal triangulation of d*Delta_2 as an (E, 4) int32 edge array.

    Rows are (i1, j1, i2, j2).  Square [i,i+1]x[j,j+1] is split by the segment
    (i+1, j)-(i, j+1); the top-right triangle of a square exists only when it
    still lies in the simplex.
    """
    tris = []
    for j in range(d):
        for i in range(d - j):
            tris.append(((i, j), (i + 1, j), (i, j + 1)))
            if i + j + 2 <= d:
                tris.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    return _edges_from_triangles(tris)


def fan_triangulation(d: int) -> np.ndarray:
    """A unimodular triangulation of d*Delta_2 (d >= 2) with a vertex of high
    degree, as an (E, 4) int32 edge array: in the strip 0 <= i <= 1, (0, 0)
    is joined to every (1, j), j < d, and to (0, 1), and (1, d - 1) to every
    (0, j), j >= 1; the rest, (d-1)*Delta_2 shifted by (1, 0), is split by
    anti-diagonals.  (0, 0) then has d + 1 neighbours in each quadrant of the
    reflected triangulation, 4d in all."""
    if d < 2:
        raise ValueError("the fan triangulation needs d >= 2")
    tris = [((0, 0), (1, j), (1, j + 1)) for j in range(d - 1)]
    tris.append(((0, 0), (1, d - 1), (0, 1)))
    tris += [((0, j), (1, d - 1), (0, j + 1)) for j in range(1, d)]
    for j in range(d - 1):
        for i in range(1, d - j):
            tris.append(((i, j), (i + 1, j), (i, j + 1)))
            if i + j + 2 <= d:
                tris.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    return _edges_from_triangles(tris)


def _lifting(d: int, seed: int, tri_id: int, attempt: int) -> dict:
    base = splitmix64_int((seed * 1_000_003 + tri_id) & _MASK64)
    base = splitmix64_int(base ^ ((attempt * _GOLDEN) & _MASK64))
    w = {}
    n = 0
    for j in range(d + 1):
        for i in range(d + 1 - j):
            r = splitmix64_int((base + n) & _MASK64) % 2001
            w[(i, j)] = 1000 * (i * i + j * j + (i + j) * (i + j)) + r
            n += 1
    return w


def _lower_hull_triangulation(d: int, w: dict):
    """Exact gift-wrapping of the lower hull of {(i, j, w(i, j))}.

    Returns the list of projected facets (each a CCW triple of lattice points)
    or None when the lifting is degenerate (four lifted points coplanar on the
    lower hull) or when the induced subdivision is not a unimodular
    triangulation.
    """
    pts = sorted(w.keys())
    P = np.array([[p[0], p[1], w[p]] for p in pts], dtype=np.int64)
    index = {p: n for n, p in enumerate(pts)}

    def orient2(a, b, c):
        return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])

    def below(a, b, c, cand):
        # a, b, c CCW in the plane; returns det per candidate (<0 means below)
        ab = P[b] - P[a]
        ac = P[c] - P[a]
        ap = P[cand] - P[a]
        return (ab[0] * (ac[1] * ap[:, 2] - ac[2] * ap[:, 1])
                - ab[1] * (ac[0] * ap[:, 2] - ac[2] * ap[:, 0])
                + ab[2] * (ac[0] * ap[:, 1] - ac[1] * ap[:, 0]))

    allidx = np.arange(len(pts))

    def wrap(a, b):
        """Facet on the left of directed edge a->b, or None if a->b is on the hull."""
        o = (P[b, 0] - P[a, 0]) * (P[:, 1] - P[a, 1]) - (P[b, 1] - P[a, 1]) * (P[:, 0] - P[a, 0])
        cand = allidx[o > 0]
        if cand.size == 0:
            return None, False
        best = int(cand[0])
        for c in cand[1:]:
            c = int(c)
            if below(a, b, best, np.array([c]))[0] < 0:
                best = c
        dets = below(a, b, best, cand)
        if np.any(dets < 0):
            return None, True
        on = cand[(dets == 0)]
        if on.size != 1:
            return None, True  # degenerate: a 4th lifted point on this facet
        return best, False

    start_a, start_b = index[(0, 0)], index[(1, 0)]
    tris = set()
    stack = [(start_a, start_b)]
    done = set()
    while stack:
        a, b = stack.pop()
        if (a, b) in done:
            continue
        done.add((a, b))
        c, degenerate = wrap(a, b)
        if degenerate:
            return None
        if c is None:
            continue
        key = tuple(sorted((a, b, c)))
        if key in tris:
            continue
        tris.add(key)
        for (x, y) in ((b, c), (c, a), (a, b)):
            if (y, x) not in done:
                stack.append((y, x))
        if len(tris) > 4 * d * d:
            return None
    out = []
    used = set()
    for key in tris:
        a, b, c = key
        pa, pb, pc = pts[a], pts[b], pts[c]
        o = orient2(pa, pb, pc)
        if abs(o) != 1:
            return None
        if o < 0:
            pb, pc = pc, pb
        out.append((pa, pb, pc))
        used.update((a, b, c))
    if len(out) != d * d or len(used) != len(pts):
        return None
    return out


def regular_triangulation(d: int, seed: int, tri_id: int = 0, max_attempts: int = 1000):
    """Seeded regular unimodular triangulation of d*Delta_2 (edge array).

    Draws liftings omega = 1000*(i^2+j^2+(i+j)^2) + U_int[0,2000] until the
    lower hull projects to a unimodular triangulation.  Returns the (E, 4)
    edge array; E = 3d(d+1)/2.
    """
    if d == 1:
        return standard_triangulation(1)
    for attempt in range(max_attempts):
        tris = _lower_hull_triangulation(d, _lifting(d, seed, tri_id, attempt))
        if tris is not None:
            return _edges_from_triangles(tris)
    raise RuntimeError(f"no unimodular lifting found for d={d}")


def regular_triangulations(d: int, count: int, seed: int):
    """``count`` pairwise distinct seeded regular unimodular triangulations."""
    seen = set()
    out = []
    tri_id = 0
    while len(out) < count:
        e = regular_triangulation(d, seed, tri_id)
        tri_id += 1
        key = e.tobytes()
        if key in seen:
            continue
        seen.add(key)
        out.append(e)
        if tri_id > 100 * count + 100:
            raise RuntimeError("too many duplicate triangulations")
    return out


# ----------------------------------------------------------------------------
# sign vectors
# ----------------------------------------------------------------------------

def random_masks(n: int, d: int, seed: int, stream: int = 0) -> np.ndarray:
    """(n, W) uint64 sign words, bits >= |A| cleared; counter-based splitmix64."""
    W = sign_words(d)
    npts = num_points(d)
    base = splitmix64_int(((seed & _MASK64) * 0x100000001B3 + stream) & _MASK64)
    ctr = np.uint64(base) + np.arange(n * W, dtype=np.uint64)
    words = splitmix64(ctr).reshape(n, W)
    for w in range(W):
        nb = min(64, npts - 64 * w)
        if nb < 64:
            words[:, w] &= np.uint64((1 << nb) - 1)
    return words


def splitmix_sign_vectors(d: int, base: int, n: int) -> np.ndarray:
    """(n, W) uint64 sign vectors of the splitmix64 counters base .. base+n-1:
    word w of counter k is splitmix64(k * W + w) (mod 2^64), bits >= |A|
    cleared."""
    W = sign_words(d)
    npts = num_points(d)
    with np.errstate(over="ignore"):
        k = np.uint64(base & _MASK64) + np.arange(n, dtype=np.uint64)
        ctr = k[:, None] * np.uint64(W) + np.arange(W, dtype=np.uint64)[None, :]
    words = splitmix64(ctr)
    nb = npts - 64 * (W - 1)
    if nb < 64:
        words[:, W - 1] &= np.uint64((1 << nb) - 1)
    return words
