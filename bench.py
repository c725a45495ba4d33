"""Benchmark of the T-curve real-scheme engine on GB300.

Workload (one step): the exhaustive sweep of one 2^32 slice of sign masks of
one seeded regular unimodular triangulation of 7*Delta_2 (36 lattice points),
every instance classified by Algorithm 1 and counted in the device hash
histogram of distinct schemes, in one persistent launch (ts_enumerate).
Under torchrun every rank sweeps its own 2^32 slice (weak scaling) and the
per-rank histograms are merged at the end.

Printed (rank 0, one JSON line): schemes/s of the whole job (device-timed
with CUDA events on the launching stream), the end-to-end rate through the
public API (ts_enumerate + ts_hist_read with the host copy), the roofline of
the enumeration kernel, the CPU oracle on a bounded sample, the plain
one-launch query kernel (ts_real_schemes on materialised masks) beside the
persistent sweep, SM clocks sampled during the timed region.

The default line also carries the d = 7 stretch sweep (all 2^35 classes of
the global sign flip), the d = 4 and d = 6 plain query configurations, the
mixed-degree batch and a short serving run (Poisson job stream on the
continuous-batching server, p50/p99 job latency).  Other workloads:

  --workload mixed    the mixed-degree batch: 32 seeded triangulations for each
                      d in 5..10, sign-vector counts log-uniform in [2^10, 2^24],
                      one CUDA-graph launch per step (the fastest of one fused
                      persistent kernel and one kernel per degree), autotuned
                      tiles
  --workload serving  a longer Poisson stream: d uniform in 6..16, 2^8..2^22
                      sign vectors per job, p50/p99 latency and schemes/s

  --workload profile  a small sweep for profiler captures (--degree, --log2n,
                      --kernel, --scratch, --splitmix; --query: the plain query
                      kernel on materialised masks instead; --batch: a batch of
                      8 triangulations of that degree, --fused in one fused
                      launch); prints its rate, which is not a bench value
  --workload intpeak  the integer-issue microbenchmark alone (all instruction
                      kinds; --trips), for profiler captures

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload d7|mixed|serving|profile|intpeak]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D = 7
SLICE = 1 << 32
TRI_SEED = 7
# Algorithmic integer operations per instance at d = 7 (sign extension,
# crossing tests on the 308 edges of T^diamond, unions over non-crossed edges,
# finds on crossed edges, antipodal unions, tree and encoding).
ALG_OPS_PER_INSTANCE = 1.2e3
METRIC = "real schemes/sec at d=7 on 1 GB300 (batched vs plain), bit-exact; p50/p99 job latency"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(edges, seconds_target: float = 12.0):
    """The CPU oracle, as it stands, on a bounded sample of the same sweep."""
    import numpy as np

    import oracle
    tri = oracle.triangles(D, edges)
    cores = os.cpu_count() or 1
    n = 1 << 14
    while True:
        masks = np.arange(n, dtype=np.uint64).reshape(-1, 1)
        t0 = time.perf_counter()
        oracle.real_schemes(D, tri, masks, n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > seconds_target / 4 or n >= 1 << 26:
            break
        n <<= 2
    return {"value": n / dt, "unit": "schemes/s", "cores": cores, "kind": "oracle",
            "sample": f"masks [0, {n}) of the d=7 sweep ({dt:.1f} s)"}


def reference_arm(args):
    """--impl reference: the CPU oracle timed as a bounded-sample stand-in."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import tcurve_inputs as ti
    edges = ti.regular_triangulation(D, seed=TRI_SEED)
    tri = oracle.triangles(D, edges)
    cores = os.cpu_count() or 1
    sample = 1 << 18
    for _ in range(args.warmup):
        oracle.real_schemes(D, tri, np.arange(1 << 12, dtype=np.uint64).reshape(-1, 1), n_threads=cores)
    times = []
    for s in range(args.steps):
        masks = np.arange(s * sample, (s + 1) * sample, dtype=np.uint64).reshape(-1, 1)
        t0 = time.perf_counter()
        oracle.real_schemes(D, tri, masks, n_threads=cores)
        times.append(time.perf_counter() - t0)
    v = sample * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "schemes/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "d7_batched_sweep", "degree": D,
                       "triangulation": f"regular unimodular, lifting seed {TRI_SEED}",
                       "sample": f"{sample} consecutive masks of the sweep per step",
                       "parallelism": f"the oracle on rank 0's {cores} host cores"},
            "cpu_baseline": {"value": v, "unit": "schemes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} consecutive masks per step"},
            "e2e": {"value": v, "unit": "schemes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--workload", default="d7",
                    choices=["d7", "mixed", "serving", "profile", "intpeak"])
    ap.add_argument("--serve-seconds", type=float, default=6.0)
    # the small case of --workload profile (for ncu captures; not a bench value)
    ap.add_argument("--degree", type=int, default=D)
    ap.add_argument("--log2n", type=int, default=26)
    ap.add_argument("--kernel", default="auto", choices=["auto", "table", "specialized", "warp"])
    ap.add_argument("--scratch", default="auto", choices=["auto", "shared", "global"])
    ap.add_argument("--splitmix", action="store_true")
    ap.add_argument("--occupancy", type=int, default=0)
    ap.add_argument("--query", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--fused", action="store_true")
    ap.add_argument("--trips", type=int, default=1 << 15)
    ap.add_argument("--no-stretch", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--families", action="store_true")
    ap.add_argument("--occupancies", default="0")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "profile":
        return profile_case(args)
    if args.workload == "intpeak":
        return intpeak_workload(args)
    if args.workload == "mixed":
        return mixed_workload(args)
    if args.workload == "serving":
        return serving_workload(args, seconds=max(args.serve_seconds, 20.0))

    import numpy as np
    import torch

    import paper_2604_09221_gb300 as eng
    import tcurve_inputs as ti
    from paper_2604_09221_gb300 import build as _b

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    _b.build()
    edges = ti.regular_triangulation(D, seed=TRI_SEED)
    tri = eng.Triangulation(D, edges)
    hist = eng.Histogram(4096, tri.code_words)
    stream = torch.cuda.current_stream()
    lo = rank * SLICE
    # the slice of rank r: masks [r 2^32, (r+1) 2^32) of the 2^36 masks
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        hist.clear(stream)
        eng.enumerate_schemes(tri, lo, lo + SLICE, hist, stream=stream)

    tri.prepare()  # build the specialised kernels before anything is timed
    int_peak = measure_int_peak(eng, args.trips)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, L2 flushed between steps ----
    clocks = ClockSampler(local)
    clocks.start()
    times, ktimes = [], []
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hist.clear(stream)
        m.record(stream)
        eng.enumerate_schemes(tri, lo, lo + SLICE, hist, stream=stream)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        ktimes.append(m.elapsed_time(b))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    codes, counts, failed = hist.read(stream)
    assert failed == 0 and int(counts.sum()) == SLICE, "sweep lost instances"
    ms = sum(times) / len(times)
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * SLICE / (ms / 1e3)

    # ---- end to end through the public API (host read of the histogram) ----
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist.clear(stream)
        eng.enumerate_schemes(tri, lo, lo + SLICE, hist, stream=stream)
        hist.read(stream)
        e2e_times.append(time.perf_counter() - t0)
    d2h = hist_read_bytes(hist, len(codes))
    e2e_ms = 1e3 * sum(e2e_times) / len(e2e_times)
    if pg:
        t = torch.tensor([e2e_ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # ---- merge of the per-rank histograms (the only exchange step) ----
    if pg:
        from paper_2604_09221_gb300 import sweep
        mine = {eng.code_to_int(c): int(k) for c, k in zip(codes, counts)}
        merged = sweep.all_gather_histogram(pg, mine, tri.code_words, device="cuda")
        if rank == 0:
            assert sum(merged.values()) == ws * SLICE

    if rank != 0:
        pg.destroy_process_group()
        return 0

    peak_tops = int_peak["peak"] / 1e12
    kms = sum(ktimes) / len(ktimes)
    achieved_tops = ALG_OPS_PER_INSTANCE * SLICE / (kms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "tc_enumerate_blocks (specialised to the triangulation)",
                "kernel_ms": kms,
                "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved_tops / peak_tops, "traffic": None,
                "traffic_note": "no input is read; DRAM carries only scratch write-backs from L2 "
                                "(55.6 MB per 2^26-mask launch by ncu), which do not scale with the "
                                "masks swept, so no per-launch figure is given for 2^32",
                "peak_source": "measured: ts_int_issue_peak, the best of its instruction kinds "
                               f"({int_peak['best']}) on this GPU in this run",
                "int_peak_tops": {k: v / 1e12 for k, v in int_peak["kinds"].items()},
                "alg_ops_per_instance": ALG_OPS_PER_INSTANCE}
    line = {"metric": METRIC, "value": value, "unit": "schemes/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "d7_batched_sweep", "degree": D, "slice": SLICE,
                       "triangulation": f"regular unimodular, lifting seed {TRI_SEED}",
                       "parallelism": f"range-sharded x{ws}",
                       "l2": "256 MiB buffer written between steps (outside the event-timed region); "
                             "the sweep reads no HBM input",
                       "wall_s": wall},
            "distinct_schemes": len(codes),
            "e2e": {"value": ws * SLICE / (e2e_ms / 1e3), "unit": "schemes/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
            # per step: ts_hist_clear's kernel and one enumeration kernel
            "gpu_launches": 2 * args.steps,
            "roofline": roofline, "clocks": clk}
    if not args.no_plain:
        line["plain"] = plain_kernel(eng, tri, ti, stream)
    if not args.no_stretch:
        line["stretch"] = stretch_sweep(eng, tri, stream)
    if not args.no_configs:
        line["configs"] = configs_run(eng, ti, stream)
    if not args.no_mixed:
        mx = mixed_run(args.steps, args.warmup)
        mx["alg_frac"] = mx["alg_tops"] * 1e12 / int_peak["peak"]
        line["mixed"] = mx
    if not args.no_serving:
        line["serving"] = serving_run(args.serve_seconds)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(edges)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def configs_run(eng, ti, stream):
    """The two plain query configurations, timed with CUDA events:
    d4_plain: all 2^15 sign vectors of the anti-diagonal triangulation of
    4*Delta_2 (one u64 word each; bit 1 = a -1 coefficient) in one
    ts_real_schemes launch (median of 5); d6_plain: 64 seeded regular
    triangulations of 6*Delta_2, 2^20 materialised splitmix64 sign vectors
    each (512 MiB of sign words in all), either one table-driven
    ts_real_schemes launch per triangulation or one fused batch launch over
    all 64 (jobs reading those sign vectors), each timed as a whole (median
    of 3); the faster is reported, both are listed."""
    import torch

    def med(fn, reps):
        out = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    t4 = eng.Triangulation(4, ti.standard_triangulation(4))
    n4 = 1 << 15
    m4 = torch.arange(n4, dtype=torch.int64, device="cuda")
    o4 = torch.empty((n4, 1), dtype=torch.int64, device="cuda")
    f4 = lambda: t4.real_schemes(m4, out=o4, stream=stream, sync=False)  # noqa: E731
    f4()
    ms4 = med(f4, 5)
    t4.sync(stream)
    tris = [eng.Triangulation(6, e) for e in ti.regular_triangulations(6, 64, seed=6)]
    n6 = 1 << 20
    masks = [eng.splitmix_masks(6, k << 20, n6, stream=stream) for k in range(64)]
    outs = [torch.empty((n6, 1), dtype=torch.int64, device="cuda") for _ in range(64)]
    for t in tris:
        t.set_kernel(eng.TS_KERNEL_TABLE)

    def f6():
        for t, m, o in zip(tris, masks, outs):
            t.real_schemes(m, out=o, stream=stream, sync=False)
    f6()
    ms6 = med(f6, 3)
    for t in tris:
        t.sync(stream)
    # the same 64 x 2^20 sign vectors as one batch in one fused launch (each
    # job reads its sign vectors, writes their codes and its histogram)
    batch = eng.Batch(tris, [n6] * 64, [k << 20 for k in range(64)], code_outputs=outs,
                      hist_capacity=1024)
    for k, m in enumerate(masks):
        batch.set_signs(k, m)
    batch.set_fused(True)
    fb = lambda: batch.run(graph=True, stream=stream)  # noqa: E731
    fb()
    ms6f = med(fb, 3)
    for k in range(64):
        codes, cnt, failed = batch.read(k, stream=stream)
        assert failed == 0 and int(cnt.sum()) == n6
    batch.close()
    fused = ms6f < ms6
    return {"d4_plain": {"sign_vectors": n4, "ms": ms4, "value": n4 / (ms4 / 1e3),
                         "unit": "schemes/s", "launches": 1},
            "d6_plain": {"triangulations": 64, "sign_vectors": 64 * n6, "ms": min(ms6, ms6f),
                         "value": 64 * n6 / (min(ms6, ms6f) / 1e3), "unit": "schemes/s",
                         "launches": 1 if fused else 64, "hbm_bytes": 64 * n6 * 16,
                         "kernel": "table-driven",
                         "plan": "one fused batch launch" if fused else "one launch per triangulation",
                         "plan_ms": {"per_triangulation": ms6, "fused_batch": ms6f}}}


def measure_int_peak(eng, trips):
    """The integer-issue peak measured on this GPU now: lane operations per
    second of each instruction kind of ts_int_issue_peak (best of two runs),
    and the best kind, which is the roofline's denominator."""
    kinds = {}
    for k, name in eng.INT_PEAK_KINDS.items():
        kinds[name] = max(eng.int_issue_peak(k, trips)[0] for _ in range(2))
    best = max(kinds, key=kinds.get)
    return {"kinds": kinds, "best": best, "peak": kinds[best]}


def stretch_sweep(eng, tri, stream):
    """All 2^35 masks of the d = 7 triangulation modulo the global sign flip
    (TS_ENUM_FLIP: the 2^35 masks with sigma(0,0) = 0), one ts_enumerate,
    timed once with CUDA events after one 2^30 warm-up sweep."""
    import torch
    n = 1 << (tri.num_points - 1)
    h = eng.Histogram(4096, tri.code_words)
    eng.enumerate_schemes(tri, 0, 1 << 30, h, eng.TS_ENUM_FLIP, stream=stream)
    h.clear(stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    eng.enumerate_schemes(tri, 0, n, h, eng.TS_ENUM_FLIP, stream=stream)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    codes, counts, failed = h.read(stream)
    assert failed == 0 and int(counts.sum()) == n, "stretch sweep lost instances"
    assert len(codes) <= 121, "more than the 121 real schemes of degree 7"
    return {"workload": "d7_flip_sweep_2p35", "masks": n, "ms": ms,
            "value": n / (ms / 1e3), "unit": "schemes/s", "distinct_schemes": len(codes),
            "flags": "TS_ENUM_FLIP"}


def intpeak_workload(args):
    """The integer-issue microbenchmark alone (for profiler captures)."""
    import torch

    import paper_2604_09221_gb300 as eng
    from paper_2604_09221_gb300 import build as _b
    torch.cuda.set_device(0)
    _b.build()
    r = measure_int_peak(eng, args.trips)
    print(json.dumps({"intpeak": True, "trips": args.trips,
                      "tops": {k: v / 1e12 for k, v in r["kinds"].items()}, "best": r["best"]}),
          flush=True)
    return 0


def profile_case(args):
    """A small sweep for profiler captures: masks [0, 2^log2n) of the bench's
    seeded regular triangulation of the given degree, swept twice (plain masks,
    or the splitmix64 stream for d >= 10 or with --splitmix)."""
    import torch

    import paper_2604_09221_gb300 as eng
    import tcurve_inputs as ti
    from paper_2604_09221_gb300 import build as _b
    torch.cuda.set_device(0)
    _b.build()
    d = args.degree
    tri = eng.Triangulation(d, ti.regular_triangulation(d, seed=TRI_SEED if d == D else d))
    tri.set_kernel({"auto": eng.TS_KERNEL_AUTO, "table": eng.TS_KERNEL_TABLE,
                    "specialized": eng.TS_KERNEL_SPECIALIZED, "warp": eng.TS_KERNEL_WARP}[args.kernel])
    tri.set_scratch({"auto": eng.TS_SCRATCH_AUTO, "shared": eng.TS_SCRATCH_SHARED,
                     "global": eng.TS_SCRATCH_GLOBAL}[args.scratch])
    tri.set_occupancy(args.occupancy)
    if args.kernel in ("auto", "specialized") and d <= 9:
        tri.prepare()
    n = 1 << args.log2n
    if args.batch:  # a one-degree batch of 8 triangulations, n sign vectors in all
        tris8 = [eng.Triangulation(d, e) for e in ti.regular_triangulations(d, 8, seed=31 + d)]
        batch = eng.Batch(tris8, [n // 8] * 8, [job_base(3100 + d, k) for k in range(8)])
        batch.set_kernel(d, {"auto": eng.TS_KERNEL_AUTO, "table": eng.TS_KERNEL_TABLE,
                             "specialized": eng.TS_KERNEL_SPECIALIZED}[args.kernel])
        if args.fused:  # the fused launch, thread tiles of 1024 sign vectors
            batch.set_fused(True)
        ms = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            batch.run(graph=False)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        for j in range(8):
            codes, cnt, failed = batch.read(j)
            assert failed == 0 and int(cnt.sum()) == n // 8
        info = batch.info(d)
        info.pop("log")
        print(json.dumps({"profile_case": True, "batch": True, "fused": args.fused, "degree": d,
                          "n": n, "ms": ms,
                          "info": info, "schemes_per_s": n / (min(ms) / 1e3)}), flush=True)
        return 0
    if args.query:  # the plain query kernel on n materialised sign vectors
        masks = eng.splitmix_masks(d, 0, n)
        out = torch.empty((n, tri.code_words), dtype=torch.int64, device="cuda")
        ms = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            tri.real_schemes(masks, out=out, sync=False)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        tri.sync()
        print(json.dumps({"profile_case": True, "query": True, "degree": d, "n": n,
                          "kernel": args.kernel, "ms": ms,
                          "bytes_per_launch": n * 8 * (tri.sign_words + tri.code_words),
                          "schemes_per_s": n / (min(ms) / 1e3)}), flush=True)
        return 0
    flags = eng.TS_ENUM_SPLITMIX if (args.splitmix or d > 9) else 0
    h = eng.Histogram(1 << 14, tri.code_words)
    ms = []
    for _ in range(2):
        h.clear()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        eng.enumerate_schemes(tri, 0, n, h, flags)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    codes, counts, failed = h.read()
    assert failed == 0 and int(counts.sum()) == n
    print(json.dumps({"profile_case": True, "degree": d, "n": n, "kernel": args.kernel,
                      "scratch": args.scratch, "occupancy": args.occupancy,
                      "splitmix": bool(flags), "ms": ms,
                      "schemes_per_s": n / (min(ms) / 1e3), "distinct": len(counts)}), flush=True)
    return 0


def hist_read_bytes(hist, n_codes):
    """Bytes ts_hist_read copies to the host: the number of packed entries,
    the error word, the failure counter, then the packed codes and counts."""
    return int(8 + 4 + 8 + n_codes * (8 * hist.code_words + 8))


def plain_kernel(eng, tri, ti, stream):
    """The plain one-launch query kernel on materialised masks (same slice)."""
    import numpy as np
    import torch
    n = 1 << 26
    masks = torch.arange(n, dtype=torch.int64, device="cuda").reshape(-1, 1)
    out = torch.empty((n, tri.code_words), dtype=torch.int64, device="cuda")
    tri.real_schemes(masks, out=out, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tri.real_schemes(masks, out=out, stream=stream, sync=False)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    tri.sync(stream)
    ms = statistics.median(times)
    nbytes = n * 8 * (tri.sign_words + tri.code_words)  # sign words in, code words out
    hbm_peak = measured_peaks().get("hbm_gbs")
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"value": n / (ms / 1e3), "unit": "schemes/s",
            "kernel": "tc_real_schemes (specialised, one launch over materialised masks)",
            "n": n, "ms": ms, "hbm_bytes": nbytes, "hbm_gbs": gbs,
            "hbm_frac": gbs / hbm_peak if hbm_peak else None,
            "hbm_peak_gbs": hbm_peak}


def job_base(seed, stream):
    import tcurve_inputs as ti
    m = (1 << 64) - 1
    return ti.splitmix64_int(((seed & m) * 0x100000001B3 + stream) & m)


def serving_run(seconds, degrees=tuple(range(6, 17)), per_degree=4, slots=8, seed=2027):
    """Poisson stream of jobs on the continuous-batching server, d uniform in
    `degrees` over resident triangulations (table-driven kernels, nothing
    compiled) and histograms.  Job kinds: half are sampled jobs (2^U(8,22)
    splitmix64 sign vectors, one in eight also returning codes), a quarter
    query jobs (2^U(8,18) caller sign vectors from host memory, codes back),
    a quarter exhaustive enumeration ranges (2^U(8,22) masks, flags 0,
    TS_ENUM_FLIP or TS_ENUM_REDUCED).  The arrival rate is 70 % of the
    capacity measured on a closed burst.  Latency percentiles per kind."""
    import numpy as np
    import torch

    import paper_2604_09221_gb300 as eng
    import tcurve_inputs as ti
    from paper_2604_09221_gb300.serve import GpuExecutor, Job, Server, percentile
    tris = [eng.Triangulation(d, e) for d in degrees
            for e in ti.regular_triangulations(d, per_degree, seed=seed + d)]
    ex = GpuExecutor(tris, slots=slots, kernel=eng.TS_KERNEL_TABLE)
    rng = np.random.default_rng(seed)
    flag_set = (0, eng.TS_ENUM_FLIP, eng.TS_ENUM_REDUCED)

    def draw():
        t = int(rng.integers(0, len(tris)))
        u = rng.uniform()
        if u < 0.5:
            return Job(tri=t, n=int(2 ** rng.uniform(8, 22)), base=int(rng.integers(0, 1 << 62)),
                       want_codes=bool(rng.uniform() < 0.125))
        if u < 0.75:
            n = int(2 ** rng.uniform(8, 18))
            return Job(tri=t, kind="query",
                       signs=ti.random_masks(n, tris[t].d, int(rng.integers(0, 1 << 30))))
        lo = int(rng.integers(0, 1 << 24))
        return Job(tri=t, kind="enum", lo=lo, hi=lo + int(2 ** rng.uniform(8, 22)),
                   flags=flag_set[int(rng.integers(0, 3))])

    srv = Server(ex, slots=slots, mem_budget=1 << 32)
    for f in [srv.submit(draw()) for _ in range(2 * slots)]:
        f.result()
    burst = [draw() for _ in range(64)]
    t0 = time.perf_counter()
    for f in [srv.submit(j) for j in burst]:
        f.result()
    cap_jobs = len(burst) / (time.perf_counter() - t0)
    rate = 0.7 * cap_jobs
    srv.completed.clear()
    jobs, futs = [], []
    t_start = time.perf_counter()
    t_next = t_start
    while t_next - t_start < seconds:
        now = time.perf_counter()
        if now < t_next:
            time.sleep(min(t_next - now, 0.002))
            continue
        j = draw()
        jobs.append(j)
        futs.append(srv.submit(j))
        t_next += rng.exponential(1.0 / rate)
    res = [f.result() for f in futs]
    wall = time.perf_counter() - t_start
    srv.close()
    torch.cuda.synchronize()
    lat = [r.latency * 1e3 for r in res]
    inst = sum(j.n for j in jobs)
    kinds = {}
    for k in ("sample", "query", "enum"):
        lk = [r.latency * 1e3 for r in res if r.kind == k]
        kinds[k] = {"jobs": len(lk), "p50_ms": percentile(lk, 50), "p99_ms": percentile(lk, 99),
                    "schemes": sum(j.n for j in jobs if j.kind == k)}
    return {"jobs": len(jobs), "arrival_rate_jobs_per_s": rate, "capacity_jobs_per_s": cap_jobs,
            "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "kinds": kinds,
            "mean_queue_ms": 1e3 * sum(r.queued for r in res) / len(res),
            "schemes_per_s": inst / wall, "slots": slots, "degrees": list(degrees),
            "sign_vectors_per_job": "sample 2^U(8,22), query 2^U(8,18), enum 2^U(8,22)",
            "kernel": "table-driven (resident, uncompiled; global scratch from d = 7)",
            "resident_mb": srv.resident / 2 ** 20, "requeued": len(srv.requeued),
            "peak_running": srv.peak_running, "seconds": wall}


def serving_workload(args, seconds):
    import torch
    torch.cuda.set_device(0)
    from paper_2604_09221_gb300 import build as _b
    _b.build()
    r = serving_run(seconds)
    line = {"metric": "serving: p50/p99 job latency and schemes/s (d in 6..16)",
            "value": r["p99_ms"], "unit": "ms (p99 job latency)", "n_gpus": 1,
            "higher_is_better": False, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "serving_poisson", "degrees": r["degrees"],
                       "sign_vectors_per_job": r["sign_vectors_per_job"]},
            "serving": r}
    print(json.dumps(line), flush=True)
    return 0


def alg_ops(d: int) -> float:
    """Algorithmic integer operations per instance at degree d: sign
    extension (3 per sign word), one crossing test, about 1.5 union steps and
    one find per edge of T^diamond (6d^2 + 2d edges), 6 per antipodal pair
    and about 4 per oval of Harnack's bound M for tree and code (1187 at d = 7)."""
    W = ((d + 1) * (d + 2) // 2 + 63) // 64
    E = 6 * d * d + 2 * d
    M = (d - 1) * (d - 2) // 2 + 1
    return 3 * W + 3.5 * E + 6 * d + 4 * M


def mixed_run(steps, warmup, degrees=(5, 6, 7, 8, 9, 10), per_degree=32, seed=31):
    """The mixed-degree batch: 32 seeded triangulations per d in 5..10,
    2^U(10,24) splitmix64 sign vectors each, one CUDA-graph launch per step
    (one fused persistent kernel for all degrees, or one per degree: the
    faster plan), tiles from the autotuner; every job's histogram is checked
    to count all its sign vectors."""
    import numpy as np
    import torch

    import paper_2604_09221_gb300 as eng
    import tcurve_inputs as ti
    from paper_2604_09221_gb300 import autotune
    rng = np.random.default_rng(seed)
    tris, counts, bases = [], [], []
    for d in degrees:
        for k, e in enumerate(ti.regular_triangulations(d, per_degree, seed=seed + d)):
            tris.append(eng.Triangulation(d, e))
            counts.append(int(2 ** rng.uniform(10, 24)))
            bases.append(job_base(seed * 100 + d, k))
    t0 = time.perf_counter()
    batch = eng.Batch(tris, counts, bases)   # compiles the specialised groups
    build_s = time.perf_counter() - t0
    # tiles cached in the file TCURVE_TILE_CACHE names, when set
    tiles = autotune.autotune(tris, counts, bases, reps=1)
    autotune.apply(batch, tiles)
    stream = torch.cuda.current_stream()

    def timed_runs(k):
        out = []
        for _ in range(k):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.run(graph=True, stream=stream)
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out
    # three launch plans, each measured on two runs; the fastest is the one
    # timed: the degree groups concurrently (forked streams), one after the
    # other, or every job of every degree in one fused persistent launch
    # (fused tiles from the autotuner)
    ftiles = autotune.autotune_fused(tris, counts, bases, reps=1)
    autotune.apply_fused(batch, ftiles)
    order = {}
    for plan in ("concurrent", "serial", "fused"):
        batch.set_fused(plan == "fused")
        batch.set_serial(plan == "serial")
        timed_runs(max(warmup, 1))
        order[plan] = min(timed_runs(2))
    plan = min(order, key=order.get)
    batch.set_fused(plan == "fused")
    batch.set_serial(plan == "serial")
    torch.cuda.synchronize()
    times = timed_runs(steps)
    for j in range(len(tris)):
        codes, cnt, failed = batch.read(j)
        assert failed == 0 and int(cnt.sum()) == counts[j]
    ms = sum(times) / len(times)
    total = sum(counts)
    ops = sum(n * alg_ops(t.d) for t, n in zip(tris, counts))
    fam = {d: batch.info(d) for d in degrees}
    return {"value": total / (ms / 1e3), "unit": "schemes/s", "ms": ms, "steps": steps,
            "workload": "mixed_degree_batch", "degrees": list(degrees),
            "triangulations_per_degree": per_degree, "jobs": len(tris), "sign_vectors": total,
            "counts": "2^U(10,24) per triangulation",
            "kernels": {str(d): fam[d]["kernel"] for d in degrees},
            "tiles": {str(d): [fam[d]["threads"], fam[d]["chunk"], fam[d]["scratch"]] for d in degrees},
            "build_s": build_s, "alg_tops": ops / (ms / 1e3) / 1e12,
            "launch": {"concurrent": "one persistent kernel per degree, concurrent streams",
                       "serial": "one persistent kernel per degree, one after the other",
                       "fused": "one fused persistent kernel for all degrees"}[plan],
            "plan_ms": order,
            "fused_tiles": {str(d): [{1: "thread", 3: "warp"}.get(k, k), c]
                            for d, (k, c) in sorted(ftiles.items())},
            "gpu_launches_per_step": 1 if plan == "fused" else len(degrees)}


def mixed_families(reps=3, degrees=(5, 6, 7, 8, 9, 10), per_degree=32, seed=31, occupancies=(0,)):
    """Each degree group of the mixed batch alone, table-driven and
    specialised (default tiles; for each register budget in `occupancies`,
    resident blocks per SM, 0 the default): schemes/s and the launch's
    resources."""
    import numpy as np
    import torch

    import paper_2604_09221_gb300 as eng
    import tcurve_inputs as ti
    rng = np.random.default_rng(seed)
    out = {}
    for d in degrees:
        tris, counts, bases = [], [], []
        for k, e in enumerate(ti.regular_triangulations(d, per_degree, seed=seed + d)):
            tris.append(eng.Triangulation(d, e))
            counts.append(int(2 ** rng.uniform(10, 24)))
            bases.append(job_base(seed * 100 + d, k))
        batch = eng.Batch(tris, counts, bases)
        row = {}
        runs = [(eng.TS_KERNEL_TABLE, 0)] + [(eng.TS_KERNEL_SPECIALIZED, o) for o in occupancies]
        for fam, occ in runs:
            for t in tris:
                t.set_occupancy(occ)
            batch.set_kernel(d, eng.TS_KERNEL_TABLE)
            batch.set_kernel(d, fam)
            batch.run(graph=False)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                batch.run(graph=False)
                b.record()
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            info = batch.info(d)
            info.pop("log")
            key = info["kernel"] + (f"_occ{occ}" if occ else "")
            row[key] = dict(info, schemes_per_s=sum(counts) / (best / 1e3), ms=best)
        out[str(d)] = row
        batch.close()
    return out


def mixed_workload(args):
    """The mixed-degree batch as one CUDA-graph launch per step (its own line)."""
    import torch

    from paper_2604_09221_gb300 import build as _b
    torch.cuda.set_device(0)
    _b.build()
    import paper_2604_09221_gb300 as eng
    if args.families:
        occ = tuple(int(x) for x in args.occupancies.split(","))
        print(json.dumps({"mixed_families": mixed_families(occupancies=occ)}), flush=True)
        return 0
    peak = measure_int_peak(eng, args.trips)
    r = mixed_run(args.steps, args.warmup)
    line = {"metric": "mixed-degree batch: schemes/s (one CUDA graph launch per step)",
            "value": r["value"], "unit": "schemes/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "dtype": "u64",
            "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "degrees", "triangulations_per_degree", "jobs",
                                         "sign_vectors", "counts", "kernels", "tiles")},
            "alg_frac": r["alg_tops"] * 1e12 / peak["peak"], "build_s": r["build_s"],
            "launch": r["launch"], "plan_ms": r["plan_ms"], "fused_tiles": r["fused_tiles"],
            "gpu_launches": r["gpu_launches_per_step"] * args.steps}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
