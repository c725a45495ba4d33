"""The pins bite: plausible mistakes planted in a copy of the oracle's C
source each make the pin suite (tests/test_oracle_pins.py) fail.  CPU only.

Each mutant is one textual change of oracle/tcurve_oracle.c written into a
temporary copy of the oracle package; a child interpreter imports that copy
as ``oracle`` before pytest starts, so the pins' ``orc`` fixture runs the
mutant.  The committed oracle is never modified.  The unchanged copy and an
equivalent rewrite are run as controls and must pass.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, original text, planted text): one mistake each, in the order of the
# oracle's steps
MUTANTS = [
    # the lattice index of the sign bits, with i and j transposed
    ("lattice_index_transposed", "return j * (d + 1) - j * (j - 1) / 2 + i;",
     "return i * (d + 1) - i * (i - 1) / 2 + j;"),
    # Harnack's bound M = (d-1)(d-2)/2 + 1 with the last term dropped
    ("harnack_bound_dropped_term", "return (d - 1) * (d - 2) / 2 + 1; }",
     "return (d - 1) * (d - 2) / 2; }"),
    # Eq. 2: the sign of a reflected point
    ("eq2_wrong_coordinate", "if (x < 0) s ^= (i & 1);", "if (x < 0) s ^= (j & 1);"),
    ("eq2_dropped_term", "if (y < 0) s ^= (j & 1);", ""),
    ("eq2_flip_all", "if (x < 0) s ^= (i & 1);", "if (x < 0) s ^= 1;"),
    # T^diamond: the quadrant reflections
    ("quadrants_transposed", "qsy[4] = {1, 1, -1, -1}", "qsy[4] = {1, -1, -1, 1}"),
    # RP^2: a boundary point is identified with its antipode, not a mirror image
    ("boundary_mirror_not_antipode",
     "vid_of(c, -c->vx[a], -c->vy[a]), vid_of(c, -c->vx[b], -c->vy[b])",
     "vid_of(c, -c->vx[a], c->vy[a]), vid_of(c, -c->vx[b], c->vy[b])"),
    # one-sidedness: an odd number of boundary passages
    ("pseudoline_any_passage", "if (comps[k].jumps & 1) {", "if (comps[k].jumps > 0) {"),
    # the lift to the sphere switches sheet at every boundary passage
    ("lift_without_sheet_switch", "        sheet ^= 1;\n", "\n"),
    # the second leg of the ray starts at the antipode -x
    ("ray_second_leg_not_antipodal",
     "seg_cross(-x, -y, px, py, g->x0, g->y0, g->x1, g->y1)",
     "seg_cross(x, y, px, py, g->x0, g->y0, g->x1, g->y1)"),
    ("ray_any_crossing", "if (!bad) return count & 1;", "if (!bad) return count > 0;"),
    # the parent is the innermost container
    ("parent_outermost_container",
     "if (in[a * no + b] && depth[b] == depth[a] - 1) par[a] = b;",
     "if (in[a * no + b] && depth[b] == 0) par[a] = b;"),
    # the canonical code: descending children, MSB first, sentinel bit
    ("children_ascending", "return strcmp(*(char *const *)b, *(char *const *)a);",
     "return strcmp(*(char *const *)a, *(char *const *)b);"),
    ("bits_reversed", "int pos = nbits - 1 - b;", "int pos = b;"),
    ("no_sentinel", "    code[nbits >> 6] |= (uint64_t)1 << (nbits & 63);\n", "\n"),
    ("depth_off_by_one", "for (int b = 0; b < no; b++) depth[a] += in[a * no + b];",
     "for (int b = 0; b < no; b++) depth[a] += in[b * no + a];"),
    # the containment relation stored with its operands transposed
    ("containment_transposed", "in[a * no + b] = (char)r;", "in[b * no + a] = (char)r;"),
    # a boundary passage not counted
    ("jump_not_counted", "        C->jumps++;\n", "\n"),
    # the orientation determinant with a wrong sign on one term
    ("orientation_sign", "return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);",
     "return (bx - ax) * (cy - ay) + (by - ay) * (cx - ax);"),
    # the count of crossed edges (a statistic the hand trace pins)
    ("crossed_edges_miscounted", "for (int e = 0; e < c.ne; e++) ncr += crossed(&c, e);",
     "for (int e = 0; e < c.ne; e++) ncr += 1;"),
    # the test point of an oval at a crossed edge's midpoint instead of a
    # segment's midpoint: on the glued boundary for a boundary edge
    ("test_point_on_an_edge", "C->px = (segs[C->first].x0 + segs[C->first].x1) / 2;",
     "C->px = segs[C->first].x0;"),
]

# Equivalent rewrites that must pass: testing the first leg of the ray in
# the lower sheet and the second in the upper one tests against the other
# lift of the oval, its image under the deck transformation of the sphere
# (which swaps the sheets), and that image separates the two lifts of P
# exactly when the first lift does.
EQUIVALENT = [
    ("other_lift", "int r = g->sheet == 0 ?", "int r = g->sheet == 1 ?"),
]

CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import oracle
assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__
import pytest
sys.exit(pytest.main([sys.argv[2], "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


def run_pins(tmp, name, old, new):
    """Exit status of the pin suite on the oracle with ``old`` replaced by ``new``."""
    base = os.path.join(tmp, name)
    pkg = os.path.join(base, "oracle")
    os.makedirs(pkg)
    for f in ("__init__.py", "tcurve_oracle.c", "tcurve_oracle.h"):
        shutil.copy(os.path.join(ROOT, "oracle", f), pkg)
    src = os.path.join(pkg, "tcurve_oracle.c")
    text = open(src).read()
    if old is not None:
        assert text.count(old) == 1, name
        text = text.replace(old, new)
        with open(src, "w") as f:
            f.write(text)
    # the planted source must still compile (a mistake, not a syntax error)
    so = os.path.join(base, "check.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-w",
                           "-o", so, src])
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", CHILD, base, PINS], cwd=base, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
    return p.returncode, p.stdout[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    jobs = [("control", None, None)] + EQUIVALENT + MUTANTS
    with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
        res = dict(zip([j[0] for j in jobs],
                       ex.map(lambda j: run_pins(str(tmp_path), *j), jobs)))
    for name in ["control"] + [e[0] for e in EQUIVALENT]:
        rc, out = res.pop(name)
        assert rc == 0, (name, out)          # unchanged or equivalent: every pin passes
    survivors = {n: out for n, (rc, out) in res.items() if rc != 1}
    assert not survivors, survivors          # rc 1: some pin failed
