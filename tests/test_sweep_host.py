"""Host logic of sharded and checkpointed sweeps, on CPU: the shards cover the
range exactly; two gloo ranks that sweep their shards (with the CPU oracle as
the chunk function) merge to the histogram of the whole range; a sweep that
stops after some chunks resumes from its checkpoint to the same result."""
import collections
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import tcurve_inputs as ti
from paper_2604_09221_gb300 import sweep


def oracle_chunk_fn(d, edges):
    import oracle
    tri = oracle.triangles(d, edges)

    def run(lo, hi):
        codes = oracle.real_schemes(d, tri, np.arange(lo, hi, dtype=np.uint64).reshape(-1, 1), n_threads=2)
        return dict(collections.Counter(int(c) for c in codes[:, 0].tolist()))
    return run


@pytest.mark.parametrize("lo,hi,world", [(0, 10, 3), (5, 6, 4), (7, 1000, 7), (0, 0, 2)])
def test_shards_cover_the_range(lo, hi, world):
    parts = [sweep.shard_range(lo, hi, r, world) for r in range(world)]
    assert parts[0][0] == lo and parts[-1][1] == hi
    for (a, b), (c, _) in zip(parts, parts[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, d, lo, hi, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    edges = ti.standard_triangulation(d)
    a, b = sweep.shard_range(lo, hi, rank, world)
    mine = oracle_chunk_fn(d, edges)(a, b)
    merged = sweep.all_gather_histogram(dist, mine, code_words=1)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(repr(sorted(merged.items())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_full_histogram(tmp_path, orc):
    d, lo, hi, world = 5, 100, 100 + 20000, 2
    out = str(tmp_path / "merged.txt")
    mp.start_processes(_rank_main, args=(world, _free_port(), d, lo, hi, out), nprocs=world,
                       join=True, start_method="spawn")
    merged = dict(eval(open(out).read()))
    want = oracle_chunk_fn(d, ti.standard_triangulation(d))(lo, hi)
    assert merged == want and sum(merged.values()) == hi - lo


def test_checkpointed_sweep_resumes(tmp_path, orc):
    d = 5
    fn = oracle_chunk_fn(d, ti.standard_triangulation(d))
    path = str(tmp_path / "ckpt.json")
    first = sweep.CheckpointedSweep(0, 50000, 7000, path, fn, tag="d5")
    first.run(max_chunks=3)           # stops part-way, as a killed job would
    assert not first.done and first.next == 21000
    second = sweep.CheckpointedSweep(0, 50000, 7000, path, fn, tag="d5")
    assert second.next == 21000
    resumed = second.run()
    assert second.done and resumed == fn(0, 50000)
    with pytest.raises(ValueError):
        sweep.CheckpointedSweep(0, 60000, 7000, path, fn, tag="d5")


def _synthetic_hist(rank, cw):
    """Histogram of rank ``rank``: codes of ``cw`` words with the top bit of
    every word set in some of them (int64 wrap-around), shared and own keys,
    and no keys at all on rank 2."""
    import random
    if rank == 2:
        return {}
    rng = random.Random(40 + rank)
    shared = [(1 << (64 * cw - 1)) | (0xFFFF << 64) | 5, (1 << 63) | 3, 1 << (64 * (cw - 1))]
    own = [rng.getrandbits(64 * cw) | 1 for _ in range(5 + 7 * rank)]
    return {k: 1 + rng.randrange(1000) for k in shared + own}


def _rank_main_multiword(rank, world, port, cw, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    merged = sweep.all_gather_histogram(dist, _synthetic_hist(rank, cw), code_words=cw)
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(repr(sorted(merged.items())))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_merge_of_multiword_codes(tmp_path):
    cw, world = 3, 3
    out = str(tmp_path / "merged")
    mp.start_processes(_rank_main_multiword, args=(world, _free_port(), cw, out), nprocs=world,
                       join=True, start_method="spawn")
    want = sweep.merge(*[_synthetic_hist(r, cw) for r in range(world)])
    for r in range(world):   # every rank holds the whole merged histogram
        assert dict(eval(open(f"{out}.{r}").read())) == want


def test_shard_files_merge_to_the_whole_range(tmp_path, orc):
    """Shards swept by separate processes (here one after another) each keep
    a checkpoint file; merging the files gives the histogram of the whole
    range, and gaps, overlaps, unfinished shards or foreign tags are refused."""
    d, lo, hi, world = 5, 1000, 1000 + 30000, 3
    fn = oracle_chunk_fn(d, ti.standard_triangulation(d))
    paths = []
    for r in range(world):
        a, b = sweep.shard_range(lo, hi, r, world)
        path = str(tmp_path / f"shard{r}.json")
        sweep.CheckpointedSweep(a, b, 4000, path, fn, tag="d5").run()
        paths.append(path)
    assert sweep.merge_checkpoint_files(paths[::-1], lo, hi, tag="d5") == fn(lo, hi)
    with pytest.raises(ValueError, match="gap or overlap"):
        sweep.merge_checkpoint_files([paths[0], paths[2]])
    with pytest.raises(ValueError, match="gap or overlap"):       # one shard given twice
        sweep.merge_checkpoint_files(paths + [paths[1]])
    with pytest.raises(ValueError, match="end at"):
        sweep.merge_checkpoint_files(paths[:2], lo, hi)
    with pytest.raises(ValueError, match="different sweeps"):
        sweep.merge_checkpoint_files(paths, tag="d6")
    unfinished = str(tmp_path / "unfinished.json")
    a, b = sweep.shard_range(lo, hi, 1, world)
    sweep.CheckpointedSweep(a, b, 4000, unfinished, fn, tag="d5").run(max_chunks=1)
    with pytest.raises(ValueError, match="stopped at"):
        sweep.merge_checkpoint_files([paths[0], unfinished, paths[2]])
