"""Host logic of the tile autotuner (paper_2604_09221_gb300.autotune) with a
fake batch and fake timings (no GPU): the fastest tile wins, tiles the
library refuses are skipped, each degree is tuned on its own jobs only, a
specialised group is tuned over its chunk alone, and cached choices are
reused without timing."""
import json

import pytest

import paper_2604_09221_gb300 as eng
from paper_2604_09221_gb300 import autotune


class FakeTri:
    def __init__(self, d):
        self.d = d


class FakeBatch:
    """Records what the tuner asks of a batch; tiles with more than 192
    threads at global scratch are refused like a tile that does not fit.
    Degrees in ``specialized`` report specialised code (128 threads, global
    scratch fixed)."""
    made = []
    specialized = set()

    def __init__(self, tris, counts, bases):
        self.tris, self.counts, self.bases = list(tris), list(counts), list(bases)
        self.degrees = sorted({t.d for t in tris})
        self.tile = None
        self.tiles = {}
        FakeBatch.made.append(self)

    def info(self, d):
        if d in FakeBatch.specialized:
            return {"kernel": "specialized", "threads": 128, "chunk": 2048, "scratch": "global",
                    "log": ""}
        return {"kernel": "table", "threads": 64, "chunk": 512, "scratch": "shared", "log": ""}

    def set_tile(self, d, threads, chunk, scratch=0):
        if scratch == autotune.GLOBAL and threads > 192:
            raise eng.TSError(1, "ts_batch_set_tile")
        if d in FakeBatch.specialized and (threads != 128 or scratch == autotune.SHARED):
            raise eng.TSError(1, "ts_batch_set_tile")
        self.tile = (threads, chunk, scratch)
        self.tiles[d] = self.tile

    def close(self):
        pass


def fake_ms(batch, reps):
    """Fastest at 128 threads, 16 vectors per thread, global scratch; d = 5
    (shared scratch only) fastest at 96 threads, 64 per thread."""
    t, c, s = batch.tile
    d = batch.degrees[0]
    if d < 8:
        return abs(t - 96) + abs(c // t - 64) / 10 + 1.0
    return abs(t - 128) + abs(c // t - 16) / 10 + (0.0 if s == autotune.GLOBAL else 5.0) + 1.0


@pytest.fixture
def fakes(monkeypatch):
    FakeBatch.made = []
    FakeBatch.specialized = set()
    timed = []

    def timer(batch, reps):
        timed.append(batch.tile)
        return fake_ms(batch, reps)

    monkeypatch.setattr(eng, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "_time_batch", timer)
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "FakeGPU")
    return timed


def test_tune_degree_picks_the_fastest_fitting_tile(fakes):
    t, c, s, ms = autotune.tune_degree([FakeTri(10)] * 2, [100, 200], [0, 1])
    assert (t, c, s) == (128, 128 * 16, autotune.GLOBAL)
    # every shared tile and the global tiles that fit were timed
    n_threads, n_chunk = len(autotune.THREADS), len(autotune.CHUNK_PER_THREAD)
    fit_global = len([x for x in autotune.THREADS if x <= 192])
    assert len(fakes) == n_threads * n_chunk + fit_global * n_chunk
    assert all(tile[2] != autotune.GLOBAL or tile[0] <= 192 for tile in fakes)


def test_small_degrees_time_shared_scratch_only(fakes):
    t, c, s, _ = autotune.tune_degree([FakeTri(5)], [100], [0])
    assert (t, c, s) == (96, 96 * 64, autotune.SHARED)
    assert {tile[2] for tile in fakes} == {autotune.SHARED}


def test_autotune_tunes_degrees_apart_and_reuses_the_cache(fakes, tmp_path):
    tris = [FakeTri(5), FakeTri(10), FakeTri(5), FakeTri(10), FakeTri(10)]
    counts, bases = [10, 20, 30, 40, 50], [1, 2, 3, 4, 5]
    cache = str(tmp_path / "tiles.json")
    tiles = autotune.autotune(tris, counts, bases, cache=cache)
    assert tiles == {5: (96, 96 * 64, autotune.SHARED), 10: (128, 128 * 16, autotune.GLOBAL)}
    # one sub-batch per degree, holding only that degree's jobs in order
    subs = {b.degrees[0]: b for b in FakeBatch.made}
    assert subs[5].counts == [10, 30] and subs[5].bases == [1, 3]
    assert subs[10].counts == [20, 40, 50] and subs[10].bases == [2, 4, 5]
    store = json.load(open(cache))
    assert set(store) == {"FakeGPU|d=5|table|tile3", "FakeGPU|d=10|table|tile3"}
    # a second run takes every tile from the cache without timing (it still
    # makes the sub-batches, whose kernel family is part of the key)
    fakes.clear()
    FakeBatch.made = []
    assert autotune.autotune(tris, counts, bases, cache=cache) == tiles
    assert fakes == [] and len(FakeBatch.made) == 2


def test_specialised_groups_tune_the_chunk_only(fakes, tmp_path):
    FakeBatch.specialized = {10}
    t, c, s, _ = autotune.tune_degree([FakeTri(10)] * 2, [100, 200], [0, 1])
    assert (t, c, s) == (128, 128 * 16, autotune.GLOBAL)
    assert fakes == [(128, 128 * k, autotune.GLOBAL) for k in autotune.CHUNK_PER_THREAD]
    cache = str(tmp_path / "tiles.json")
    autotune.autotune([FakeTri(5), FakeTri(10)], [1, 2], [0, 0], cache=cache)
    assert set(json.load(open(cache))) == {"FakeGPU|d=5|table|tile3",
                                           "FakeGPU|d=10|specialized|tile3"}


def test_apply_sets_only_the_degrees_of_the_batch():
    b = FakeBatch([FakeTri(6), FakeTri(9)], [1, 1], [0, 0])
    autotune.apply(b, {6: (64, 256, 1), 9: (128, 2048, 2), 12: (32, 32, 2)})
    assert b.tiles == {6: (64, 256, 1), 9: (128, 2048, 2)}


class FakeFusedBatch(FakeBatch):
    """A fused sub-batch: records fused tiles; refuses chunks above 4096
    like a launch that does not fit."""

    def __init__(self, tris, counts, bases):
        super().__init__(tris, counts, bases)
        self.fused = False

    def set_fused(self, fused):
        self.fused = bool(fused)

    def set_fused_tile(self, d, kind, chunk):
        if chunk > 4096:
            raise eng.TSError(1, "ts_batch_set_fused_tile")
        self.tile = (kind, chunk)
        self.tiles[d] = self.tile


def fused_ms(batch, reps):
    """Warp tiles fastest at d = 13, thread tiles with 1024 per item below."""
    assert batch.fused
    kind, chunk = batch.tile
    d = batch.degrees[0]
    if d >= 13:
        return 1.0 + (0.0 if kind == eng.TS_KERNEL_WARP else 3.0) + abs(chunk - 256) / 1e4
    return 1.0 + (0.0 if kind == eng.TS_KERNEL_TABLE else 3.0) + abs(chunk - 1024) / 1e4


def test_fused_tiles_per_degree_with_cache(monkeypatch, tmp_path):
    """autotune_fused: each degree tuned alone in a fused sub-batch; warp
    tiles offered from d = 7 only; refused tiles skipped; the cache is keyed
    by the fused family and reused without timing."""
    FakeBatch.made = []
    timed = []

    def timer(batch, reps):
        timed.append((batch.degrees[0], batch.tile))
        return fused_ms(batch, reps)

    monkeypatch.setattr(eng, "Batch", FakeFusedBatch)
    monkeypatch.setattr(autotune, "_time_batch", timer)
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "FakeGPU")
    tris = [FakeTri(5), FakeTri(13), FakeTri(5)]
    cache = str(tmp_path / "tiles.json")
    tiles = autotune.autotune_fused(tris, [10, 20, 30], [0, 1, 2], cache=cache, reps=1)
    assert tiles == {5: (eng.TS_KERNEL_TABLE, 1024), 13: (eng.TS_KERNEL_WARP, 256)}
    assert all(b.degrees in ([5], [13]) and b.fused for b in FakeBatch.made)
    assert all(k == eng.TS_KERNEL_TABLE for d, (k, c) in timed if d == 5)
    assert all(c <= 4096 for _, (k, c) in timed)          # 128 x 64 was refused
    stored = json.load(open(cache))
    assert set(stored) == {"FakeGPU|d=5|fused|tile2", "FakeGPU|d=13|fused|tile2"}
    n = len(timed)
    assert autotune.autotune_fused(tris, [10, 20, 30], [0, 1, 2], cache=cache) == tiles
    assert len(timed) == n                                # served from the cache
    applied = FakeFusedBatch(tris, [1, 1, 1], [0, 0, 0])
    autotune.apply_fused(applied, tiles)
    assert applied.tiles == tiles
