"""Write the oracle's histogram of the degree-7 sweep that bench.py times.

The bench sweeps masks [0, 2^32) of the seeded regular unimodular
triangulation ``tcurve_inputs.regular_triangulation(7, seed=7)``: every mask k
is the sign vector sigma with bit k(i, j) = sigma(i, j) (Sec. 2), and the
output is the number of masks of each real scheme (the exhaustive check of
Sec. 3).  This script computes that histogram with the CPU oracle alone
(``oracle/``; nothing of the engine is imported) and writes

  d7_seed7_sweep_2p32.hist   header lines "# ..." (the triangulation's edges,
                             the range), then one "code count" per scheme,
                             sorted by code

so that a GPU test can compare the engine's 2^32 histogram with it bin by bin.

It takes about an hour on 8 host cores.  Progress is kept in a checkpoint
file (default: in the system's temporary directory), so an interrupted run
resumes where it stopped:

    python tests/golden/make_d7_sweep_histogram.py [--threads N] [--checkpoint PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

D = 7
SEED = 7
TOTAL = 1 << 32
CHUNK = 1 << 24
OUT = os.path.join(HERE, "d7_seed7_sweep_2p32.hist")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--checkpoint",
                    default=os.path.join(tempfile.gettempdir(), "d7_seed7_sweep_2p32.ckpt.json"))
    args = ap.parse_args()

    import oracle
    import tcurve_inputs as ti
    edges = np.asarray(ti.regular_triangulation(D, seed=SEED), dtype=np.int64)
    tri = oracle.triangles(D, edges)
    edge_rows = sorted(tuple(int(x) for x in r) for r in edges.reshape(-1, 4))

    state = {"edges": edge_rows, "done": 0, "hist": {}}
    if os.path.exists(args.checkpoint):
        with open(args.checkpoint) as f:
            old = json.load(f)
        if [tuple(r) for r in old["edges"]] == edge_rows:
            state = old
    hist = {int(k): int(v) for k, v in state["hist"].items()}
    done = int(state["done"])
    t0 = time.time()
    while done < TOTAL:
        masks = np.arange(done, done + CHUNK, dtype=np.uint64).reshape(-1, 1)
        codes = oracle.real_schemes(D, tri, masks, n_threads=args.threads)[:, 0]
        u, c = np.unique(codes, return_counts=True)
        for k, v in zip(u.tolist(), c.tolist()):
            hist[k] = hist.get(k, 0) + v
        done += CHUNK
        tmp = args.checkpoint + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"edges": edge_rows, "done": done,
                       "hist": {str(k): v for k, v in hist.items()}}, f)
        os.replace(tmp, args.checkpoint)
        rate = (done - int(state["done"])) / max(time.time() - t0, 1e-9)
        print(f"{done}/{TOTAL} masks, {len(hist)} schemes, {rate:.3g} masks/s", flush=True)
    assert sum(hist.values()) == TOTAL
    with open(OUT, "w") as f:
        f.write("# Real schemes of masks [0, 2^32) of tcurve_inputs.regular_triangulation(7, seed=7),\n")
        f.write("# computed by the CPU oracle (tests/golden/make_d7_sweep_histogram.py).\n")
        f.write("# edge " + " ".join(f"{a},{b},{c},{d}" for a, b, c, d in edge_rows) + "\n")
        f.write(f"# range 0 {TOTAL}\n")
        for k in sorted(hist):
            f.write(f"{k} {hist[k]}\n")
    print(f"wrote {OUT}: {len(hist)} schemes")


if __name__ == "__main__":
    main()
