"""Exhaustive check of Fig. 2 on the GPU (manual, long: ~30 min per
triangulation on one GB300).

Fig. 2 of the paper gives, for three degree-8 triangulations, the percentage
of the 2^42 sign-distribution classes (one representative per (Z/2)^3 orbit,
Sec. 3) whose curve has k ovals, to four decimals, and the number of distinct
real schemes each realizes (123, 359 and 353).  This script sweeps all 2^42
representatives of one triangulation with ts_enumerate (TS_ENUM_REDUCED,
or with --orbits the TS_ENUM_ORBITS representatives, whose chunks keep every
middle-row pattern), checkpointing after every chunk, and compares both with
the printed values stored in this directory; --limit LOG2 only times the
first 2^LOG2 classes.

    python tests/golden/check_fig2_exhaustive.py bow_tie [checkpoint.json]

The range can also be split into N shards swept independently (one process
or machine each, every shard with its own checkpoint) and merged afterwards:

    python tests/golden/check_fig2_exhaustive.py rank015 s0.json --shard 0/4
    ...
    python tests/golden/check_fig2_exhaustive.py rank015 --merge s0.json s1.json s2.json s3.json
"""
import collections
import json
import os
import sys
import time
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SCHEMES = {"bow_tie": 123, "rank016": 359, "rank015": 353}  # Fig. 2 caption


def printed(name):
    out = {}
    with open(os.path.join(HERE, "fig2_oval_percentages.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            n, k, p = line.split()
            if n == name:
                out[int(k)] = p
    return out


def main(name, ckpt, shard=(0, 1), orbits=False, limit=None):
    import torch

    import paper_2604_09221_gb300 as eng
    from paper_2604_09221_gb300 import build, sweep
    build.build()
    torch.cuda.set_device(0)
    edges = np.loadtxt(os.path.join(HERE, f"fig2_{name}.edges"), dtype=np.int32, comments="#")
    tri = eng.Triangulation(8, edges)
    tri.prepare()
    total = 1 << 42
    flags = eng.TS_ENUM_ORBITS if orbits else eng.TS_ENUM_REDUCED
    fn = sweep.engine_chunk_fn(tri, flags=flags)
    if limit is not None:  # a timed run over the first 2^limit classes of the shard, no check
        lo, _ = sweep.shard_range(0, total, shard[0], shard[1])
        fn(lo, lo + (1 << 10))  # warm-up
        torch.cuda.synchronize()
        t = time.time()
        hist = fn(lo, lo + (1 << limit))
        torch.cuda.synchronize()
        dt = time.time() - t
        assert sum(hist.values()) == 1 << limit
        print(json.dumps({"triangulation": name, "flags": "TS_ENUM_ORBITS" if orbits else "TS_ENUM_REDUCED",
                          "classes": 1 << limit, "seconds": dt, "classes_per_s": (1 << limit) / dt,
                          "distinct_schemes": len(hist)}))
        return 0
    t0 = time.time()

    def chunk(lo, hi):
        out = fn(lo, hi)
        print(f"[{time.time() - t0:8.1f} s] {hi / total:7.2%}", file=sys.stderr, flush=True)
        return out

    lo, hi = sweep.shard_range(0, total, shard[0], shard[1])
    run = sweep.CheckpointedSweep(lo, hi, 1 << 36, ckpt, chunk,
                                  tag=name + ("/orbits" if orbits else ""))
    hist = run.run()
    assert run.done and sum(hist.values()) == hi - lo
    if shard[1] > 1:
        print(json.dumps({"triangulation": name, "shard": list(shard), "range": [lo, hi],
                          "checkpoint": ckpt, "distinct_schemes_in_shard": len(hist)}))
        return 0
    return report(name, hist, total)


def report(name, hist, total=1 << 42):
    ovals = collections.Counter()
    for code, n in hist.items():
        ovals[(code.bit_length() - 1) // 2] += n
    want = printed(name)
    rows, ok = [], True
    for k in range(23):
        # the printed figure is the percentage rounded (or cut) to 4 decimals
        exact = Fraction(100 * ovals.get(k, 0), total)
        exp = Fraction(want.get(k, "0.0000"))
        same = exp in (Fraction(round(exact * 10000), 10000), Fraction(int(exact * 10000), 10000))
        ok &= same
        rows.append((k, str(exp), float(exact), same))
    res = {"triangulation": name, "classes": total, "distinct_schemes": len(hist),
           "printed_schemes": SCHEMES[name], "oval_percentages": rows,
           "all_percentages_match": ok, "schemes_match": len(hist) == SCHEMES[name]}
    print(json.dumps(res))
    return 0 if ok and len(hist) == SCHEMES[name] else 1


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("name", nargs="?", default="bow_tie", choices=sorted(SCHEMES))
    ap.add_argument("checkpoint", nargs="?")
    ap.add_argument("--shard", default="0/1", help="r/N: sweep shard r of N")
    ap.add_argument("--merge", nargs="+", metavar="CHECKPOINT",
                    help="merge finished shard checkpoints and compare with Fig. 2")
    ap.add_argument("--orbits", action="store_true",
                    help="sweep the TS_ENUM_ORBITS representatives (the same histogram)")
    ap.add_argument("--limit", type=int, metavar="LOG2",
                    help="only time the first 2^LOG2 classes of the shard")
    a = ap.parse_args()
    if a.merge:
        from paper_2604_09221_gb300 import sweep
        tag = a.name + ("/orbits" if a.orbits else "")
        sys.exit(report(a.name, sweep.merge_checkpoint_files(a.merge, 0, 1 << 42, tag=tag)))
    r, n = (int(x) for x in a.shard.split("/"))
    sys.exit(main(a.name, a.checkpoint or f"fig2_{a.name}.ckpt.json", (r, n), a.orbits, a.limit))
