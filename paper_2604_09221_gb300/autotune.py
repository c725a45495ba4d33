"""Tile autotuner of mixed-degree batches (ts_batch).

For every degree in a batch the persistent kernel has three knobs: threads
per block, sign vectors per work item, and where the per-thread scratch
lives (shared memory, or global memory for the large degrees whose scratch
leaves few warps per SM).  A degree group that runs specialised code
(ts_batch_info: compiled per triangulation, 128-thread blocks and global
scratch fixed at compile time) has one knob, the sign vectors per work item.
The tuner times candidate tiles on the batch's own jobs of that degree (a
sub-batch, so degrees are tuned independently), keeps the fastest, and can
store the choice in a JSON cache keyed by GPU name, degree and kernel family
(path from the argument or the TCURVE_TILE_CACHE environment variable).

In the fused launch (ts_batch_set_fused: one kernel for all degrees) a
degree's tile is the kind (one thread or, from d = 7, one warp per sign
vector) and the sign vectors per work item; autotune_fused times those the
same way, on fused sub-batches of one degree.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Tuple

THREADS = (64, 96, 128, 192, 256)
CHUNK_PER_THREAD = (4, 16, 64)
SHARED, GLOBAL = 1, 2            # TS_SCRATCH_SHARED, TS_SCRATCH_GLOBAL


def scratch_choices(d: int):
    """Scratch placements worth timing: shared below d = 8, both above."""
    return (SHARED,) if d < 8 else (SHARED, GLOBAL)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _time_batch(batch, reps: int) -> float:
    import torch
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
    return best


def candidates(d: int, family: dict, threads, chunk_per_thread, scratch):
    """Tiles worth timing for a degree group of the given kernel family."""
    if family["kernel"] == "specialized":
        t = family["threads"]
        return [(t, t * c, GLOBAL) for c in chunk_per_thread]
    return [(t, t * c, s) for s in (scratch_choices(d) if scratch is None else scratch)
            for t in threads for c in chunk_per_thread]


def tune_degree(tris, counts, bases, threads: Iterable[int] = THREADS,
                chunk_per_thread: Iterable[int] = CHUNK_PER_THREAD, reps: int = 3,
                scratch: Optional[Iterable[int]] = None, sub=None) -> Tuple[int, int, int, float]:
    """Fastest (threads, chunk, scratch, ms) for the jobs (all of one degree);
    ``sub``: a batch of exactly these jobs, if one exists already."""
    from . import Batch, TSError
    d = tris[0].d
    assert all(t.d == d for t in tris)
    own = sub is None
    if own:
        sub = Batch(tris, counts, bases)
    best = None
    for t, c, s in candidates(d, sub.info(d), threads, chunk_per_thread, scratch):
        try:
            sub.set_tile(d, t, c, s)
        except TSError:
            continue  # the block does not fit shared memory
        ms = _time_batch(sub, reps)
        if best is None or ms < best[3]:
            best = (t, c, s, ms)
    if own:
        sub.close()
    if best is None:
        raise RuntimeError(f"no tile fits degree {d}")
    return best


def autotune(tris, counts, bases, cache: Optional[str] = None, reps: int = 3,
             threads: Iterable[int] = THREADS, chunk_per_thread: Iterable[int] = CHUNK_PER_THREAD
             ) -> Dict[int, Tuple[int, int, int]]:
    """Tile per degree of the batch {d: (threads, chunk, scratch)}; cached
    choices are reused, new ones stored."""
    cache = cache or os.environ.get("TCURVE_TILE_CACHE")
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
    from . import Batch
    gpu = _gpu_name()
    tiles: Dict[int, Tuple[int, int, int]] = {}
    for d in sorted({t.d for t in tris}):
        idx = [i for i, t in enumerate(tris) if t.d == d]
        sel = ([tris[i] for i in idx], [counts[i] for i in idx], [bases[i] for i in idx])
        sub = Batch(*sel)   # its kernel family decides the tile space
        key = f"{gpu}|d={d}|{sub.info(d)['kernel']}|tile3"
        if key in store:
            tiles[d] = tuple(store[key][:3])
        else:
            t, c, s, ms = tune_degree(*sel, threads, chunk_per_thread, reps, sub=sub)
            tiles[d] = (t, c, s)
            store[key] = [t, c, s, ms]
        sub.close()
    if cache:
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return tiles


def apply(batch, tiles: Dict[int, Tuple[int, ...]]):
    for d, tile in tiles.items():
        if d in batch.degrees:
            batch.set_tile(d, *tile)


# fused launch: work items of 128 x c sign vectors; warp tiles from d = 7
FUSED_THREAD_CHUNKS = (4, 8, 16, 64)
FUSED_WARP_CHUNKS = (2, 8)
FUSED_WARP_FROM = 7


def fused_candidates(d: int, thread_chunks=FUSED_THREAD_CHUNKS, warp_chunks=FUSED_WARP_CHUNKS):
    from . import TS_KERNEL_TABLE, TS_KERNEL_WARP
    out = [(TS_KERNEL_TABLE, 128 * c) for c in thread_chunks]
    if d >= FUSED_WARP_FROM:
        out += [(TS_KERNEL_WARP, 128 * c) for c in warp_chunks]
    return out


def tune_fused_degree(tris, counts, bases, reps: int = 3, thread_chunks=FUSED_THREAD_CHUNKS,
                      warp_chunks=FUSED_WARP_CHUNKS) -> Tuple[int, int, float]:
    """Fastest fused tile (kind, chunk, ms) for jobs of one degree, timed in
    a fused sub-batch of exactly these jobs."""
    from . import Batch, TSError
    d = tris[0].d
    assert all(t.d == d for t in tris)
    sub = Batch(tris, counts, bases)
    sub.set_fused(True)
    best = None
    for kind, chunk in fused_candidates(d, thread_chunks, warp_chunks):
        try:
            sub.set_fused_tile(d, kind, chunk)
        except TSError:
            continue  # the launch does not fit
        ms = _time_batch(sub, reps)
        if best is None or ms < best[2]:
            best = (kind, chunk, ms)
    sub.close()
    if best is None:
        raise RuntimeError(f"no fused tile fits degree {d}")
    return best


def autotune_fused(tris, counts, bases, cache: Optional[str] = None, reps: int = 3,
                   thread_chunks=FUSED_THREAD_CHUNKS, warp_chunks=FUSED_WARP_CHUNKS
                   ) -> Dict[int, Tuple[int, int]]:
    """Fused-launch tile per degree of the batch {d: (kind, chunk)}; cached
    choices are reused, new ones stored."""
    cache = cache or os.environ.get("TCURVE_TILE_CACHE")
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
    gpu = _gpu_name()
    tiles: Dict[int, Tuple[int, int]] = {}
    for d in sorted({t.d for t in tris}):
        idx = [i for i, t in enumerate(tris) if t.d == d]
        key = f"{gpu}|d={d}|fused|tile2"
        if key in store:
            tiles[d] = tuple(store[key][:2])
        else:
            kind, chunk, ms = tune_fused_degree([tris[i] for i in idx], [counts[i] for i in idx],
                                                [bases[i] for i in idx], reps, thread_chunks,
                                                warp_chunks)
            tiles[d] = (kind, chunk)
            store[key] = [kind, chunk, ms]
    if cache:
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return tiles


def apply_fused(batch, tiles: Dict[int, Tuple[int, int]]):
    for d, (kind, chunk) in tiles.items():
        if d in batch.degrees:
            batch.set_fused_tile(d, kind, chunk)
