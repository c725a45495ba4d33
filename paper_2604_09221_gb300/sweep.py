"""Sharded and checkpointed exhaustive sweeps (host orchestration).

The exhaustive sweep of Sec. 3 is embarrassingly parallel: every rank (one
process per GPU) sweeps a contiguous part of the index range with
``ts_enumerate`` and the only exchange is the merge of the small per-rank
histograms (at most a few thousand distinct codes) at the end.  Long sweeps
(2^42 masks of a degree-8 triangulation take hours) are run in chunks; after
each chunk the running histogram and the next index are written to a JSON
file, so a sweep that stops can resume where it stopped.  Shards run on
separate machines merge either by a collective (``all_gather_histogram``)
or from their checkpoint files (``merge_checkpoint_files``).

Everything here is host logic on top of the C ABI; the schemes themselves are
computed by the engine's kernels (or, in tests, by whatever ``chunk_fn`` the
caller passes).
"""
from __future__ import annotations

import collections
import json
import os
from typing import Callable, Dict, Optional, Tuple


def shard_range(lo: int, hi: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous part of [lo, hi) owned by ``rank`` of ``world`` ranks; the
    parts are disjoint, cover the range and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or hi < lo:
        raise ValueError("bad shard request")
    n = hi - lo
    base, extra = divmod(n, world)
    start = lo + rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def merge(*tables: Dict[int, int]) -> Dict[int, int]:
    """Key-wise sum of histograms {code: count}."""
    out: collections.Counter = collections.Counter()
    for t in tables:
        out.update(t)
    return dict(out)


def all_gather_histogram(pg, hist: Dict[int, int], code_words: int, device=None) -> Dict[int, int]:
    """Merge the histograms of all ranks of the process group ``pg`` (the
    ``torch.distributed`` module or a compatible object); every rank gets the
    merged histogram.  Works with gloo (CPU tensors) and NCCL (CUDA tensors)."""
    import torch
    world = pg.get_world_size()
    keys = sorted(hist)
    n = torch.tensor([len(keys)], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    pg.all_gather(sizes, n)
    m = max(int(s.item()) for s in sizes)
    buf = torch.zeros((max(m, 1), code_words + 1), dtype=torch.int64, device=device)
    for r, k in enumerate(keys):
        for w in range(code_words):
            word = (k >> (64 * w)) & ((1 << 64) - 1)
            buf[r, w] = word - (1 << 64) if word >= 1 << 63 else word
        buf[r, code_words] = hist[k]
    outs = [torch.zeros_like(buf) for _ in range(world)]
    pg.all_gather(outs, buf)
    merged: collections.Counter = collections.Counter()
    for o, s in zip(outs, sizes):
        for row in o[: int(s.item())].cpu().tolist():
            code = 0
            for w in range(code_words):
                code |= (row[w] & ((1 << 64) - 1)) << (64 * w)
            merged[code] += row[code_words]
    return dict(merged)


def engine_chunk_fn(tri, flags: int = 0, stream=None, capacity: int = 1 << 14):
    """A chunk function that sweeps [lo, hi) on the GPU with ts_enumerate."""
    from . import Histogram, code_to_int, enumerate_schemes
    hist = Histogram(capacity, tri.code_words)

    def run(lo: int, hi: int) -> Dict[int, int]:
        hist.clear(stream)
        enumerate_schemes(tri, lo, hi, hist, flags, stream=stream)
        codes, counts, failed = hist.read(stream)
        if failed:
            raise RuntimeError(f"{failed} instances failed in [{lo}, {hi})")
        return {code_to_int(c): int(k) for c, k in zip(codes, counts)}

    return run


def merge_checkpoint_files(paths, lo: Optional[int] = None, hi: Optional[int] = None,
                           tag: Optional[str] = None) -> Dict[int, int]:
    """Merge the checkpoint files of finished shards (one per process or
    box; ``CheckpointedSweep`` wrote them) into the histogram of the whole
    range.  The shards must carry one tag, be complete, be disjoint and cover
    [lo, hi) exactly (by default the union of their ranges, which must then
    be contiguous); otherwise ValueError."""
    shards = []
    for p in paths:
        with open(p) as f:
            st = json.load(f)
        if int(st["next"]) < int(st["hi"]):
            raise ValueError(f"{p}: shard [{st['lo']}, {st['hi']}) stopped at {st['next']}")
        shards.append((int(st["lo"]), int(st["hi"]), st.get("tag", ""), st["hist"], p))
    if not shards:
        raise ValueError("no shards")
    tags = {s[2] for s in shards}
    if len(tags) != 1 or (tag is not None and tags != {tag}):
        raise ValueError(f"shards of different sweeps: tags {sorted(tags)}")
    shards.sort(key=lambda s: (s[0], s[1]))
    lo = shards[0][0] if lo is None else lo
    hi = max(s[1] for s in shards) if hi is None else hi
    at = lo
    for a, b, _, _, p in shards:
        if a != at:
            raise ValueError(f"{p}: shard starts at {a}, expected {at} (gap or overlap)")
        at = b
    if at != hi:
        raise ValueError(f"shards end at {at}, the range at {hi}")
    return merge(*[{int(k): int(v) for k, v in s[3].items()} for s in shards])


class CheckpointedSweep:
    """Sweep [lo, hi) in chunks of ``chunk`` indices, saving the running
    histogram and the next index to ``path`` after every chunk.  Constructing
    it with an existing file of the same range resumes from the saved index."""

    def __init__(self, lo: int, hi: int, chunk: int, path: str,
                 chunk_fn: Callable[[int, int], Dict[int, int]], tag: str = ""):
        if chunk <= 0 or hi < lo:
            raise ValueError("bad sweep")
        self.lo, self.hi, self.chunk, self.path, self.fn, self.tag = lo, hi, chunk, path, chunk_fn, tag
        self.next = lo
        self.hist: Dict[int, int] = {}
        if os.path.exists(path):
            with open(path) as f:
                st = json.load(f)
            if (st["lo"], st["hi"], st.get("tag", "")) != (lo, hi, tag):
                raise ValueError(f"checkpoint {path} belongs to another sweep")
            self.next = int(st["next"])
            self.hist = {int(k): int(v) for k, v in st["hist"].items()}

    def _save(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"lo": self.lo, "hi": self.hi, "tag": self.tag, "next": self.next,
                       "hist": {str(k): v for k, v in sorted(self.hist.items())}}, f)
        os.replace(tmp, self.path)

    def run(self, max_chunks: Optional[int] = None) -> Dict[int, int]:
        """Process chunks until done (or ``max_chunks`` chunks); returns the
        histogram so far.  ``done`` tells whether the range is complete."""
        k = 0
        while self.next < self.hi and (max_chunks is None or k < max_chunks):
            end = min(self.hi, self.next + self.chunk)
            self.hist = merge(self.hist, self.fn(self.next, end))
            self.next = end
            self._save()
            k += 1
        return dict(self.hist)

    @property
    def done(self) -> bool:
        return self.next >= self.hi
