"""Test-side helpers: nesting trees <-> canonical codes, classical invariants.

A scheme is a list of top-level ovals; each oval is the list of the ovals
directly inside it.  The code format (a convention of this project, the paper
fixes none) is: enc(oval) = '1' + (children encodings in descending
lexicographic order) + '0'; the scheme's bits are the top-level encodings in
the same order; code = (1 << nbits) | bits.
"""
from __future__ import annotations


def enc(children) -> str:
    return "".join(sorted(("1" + enc(c) + "0" for c in children), reverse=True))


def code_of(children) -> int:
    b = enc(children)
    return (1 << len(b)) | (int(b, 2) if b else 0)


def tree_of(code: int):
    """Inverse of code_of; raises on malformed codes."""
    if code <= 0:
        raise ValueError("code must be positive")
    bits = bin(code)[3:]
    pos = 0

    def parse():
        nonlocal pos
        out = []
        while pos < len(bits) and bits[pos] == "1":
            pos += 1
            out.append(parse())
            if pos >= len(bits) or bits[pos] != "0":
                raise ValueError("unbalanced code")
            pos += 1
        return out

    t = parse()
    if pos != len(bits):
        raise ValueError("trailing bits")
    if enc(t) != bits:
        raise ValueError("code is not in canonical order")
    return t


def ovals(tree) -> int:
    return sum(1 + ovals(c) for c in tree)


def depth(tree) -> int:
    return max((1 + depth(c) for c in tree), default=0)


def parity_counts(tree, level=0):
    """(p, n): ovals inside an even / odd number of other ovals."""
    p = n = 0
    for c in tree:
        if level % 2 == 0:
            p += 1
        else:
            n += 1
        cp, cn = parity_counts(c, level + 1)
        p += cp
        n += cn
    return p, n


def chains(tree):
    """For every oval, the set (frozenset of ids) of ovals containing it or
    equal to it; ids are assigned in DFS order."""
    out = []
    counter = [0]

    def rec(t, anc):
        for c in t:
            me = counter[0]
            counter[0] += 1
            a = anc | {me}
            out.append(a)
            rec(c, a)

    rec(tree, frozenset())
    return out


def harnack_M(d: int) -> int:
    return (d - 1) * (d - 2) // 2 + 1


def check_classical(d: int, code: int, regular: bool = True) -> list[str]:
    """Necessary conditions on the real scheme of a T-curve of degree d.

    Harnack's bound holds for every T-curve; the others are theorems about
    real algebraic curves and apply through Thm. 1 when T is regular.
    Returns the list of violated conditions (empty if all hold)."""
    bad = []
    t = tree_of(code)
    n_ov = ovals(t)
    comps = n_ov + (d % 2)
    if comps > harnack_M(d):
        bad.append("harnack")
    if not regular:
        return bad
    # Bezout with a line through points inside two ovals X, Y: it meets every
    # oval containing X or Y at least twice, and the pseudoline once.
    ch = chains(t)
    worst = max((len(a | b) for a in ch for b in ch), default=0)
    if 2 * worst + (d % 2) > d:
        bad.append("bezout-line")
    if d % 2 == 0:
        k = d // 2
        p, n = parity_counts(t)
        if not (-(3 * k * (k - 1)) / 2 <= p - n <= (3 * k * (k - 1)) / 2 + 1):
            bad.append("petrovskii")
        if comps == harnack_M(d) and (p - n - k * k) % 8 != 0:
            bad.append("gudkov-rokhlin")
        if comps == harnack_M(d) - 1 and (p - n - k * k - 1) % 8 != 0 and (p - n - k * k + 1) % 8 != 0:
            bad.append("kharlamov-gudkov-krakhnov")
    return bad


def rohlin_viro(d: int, code: int) -> str:
    """Rohlin-Viro notation, e.g. <J + 1<1> + 2> (with '+' for the disjoint union)."""
    def part(t):
        groups = []
        for c in t:
            s = part(c)
            if groups and groups[-1][0] == s:
                groups[-1][1] += 1
            else:
                groups.append([s, 1])
        items = []
        for s, k in groups:
            items.append(f"{k}<{s}>" if s else f"{k}")
        return " + ".join(items)

    t = tree_of(code)
    inner = part(t)
    if d % 2:
        inner = "J" + (" + " + inner if inner else "")
    return f"<{inner or '0'}>"


def orbit_pivots(d: int):
    """The pivot bits (p1 > p2) of the high part of a mask for the orbit
    sweep (TS_ENUM_ORBITS), from their definition: the class group's
    elements that keep sigma(0, 1) = 0 add a + b i + c j with a = c, which on
    the high bits (lattice points with j >= 1 other than (0, 1), bit
    k(i, j) - d - 2) spans A = {i odd} and B = {j even}; the pivots are the
    leading bits of A and B in echelon form."""
    def k(i, j):
        return j * (d + 1) - j * (j - 1) // 2 + i
    a = b = 0
    for j in range(1, d + 1):
        for i in range(0, d + 1 - j):
            if (i, j) == (0, 1):
                continue
            bit = k(i, j) - d - 2
            a |= (i % 2) << bit
            b |= (1 - j % 2) << bit
    if b.bit_length() > a.bit_length():
        a, b = b, a
    if b.bit_length() == a.bit_length():
        b ^= a
    return a.bit_length() - 1, b.bit_length() - 1


def orbit_mask(d: int, k: int) -> int:
    """Mask m(k) of the orbit sweep: the middle-row pattern k mod 2^(d+1),
    bit d + 1 clear, and the high part k >> (d + 1) with zero bits inserted
    at the pivots (the lower one first)."""
    p1, p2 = orbit_pivots(d)

    def ins(x, p):
        return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1))
    t, u = k & ((1 << (d + 1)) - 1), k >> (d + 1)
    return (ins(ins(u, p2), p1) << (d + 2)) | t
