"""Multi-process host logic of the sharded forms, on CPU ranks (gloo,
world size 2): frequency bands of one plane summed on separate ranks and
gathered equal the unsplit result; the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1805_12258_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nt, n, H = 21, 5000, 8
        plane = synth.noise(nt, n, seed=44)          # every rank holds the plane
        ta = synth.thresholds(1e-3, H, nt)
        lo, hi = shard.band_bounds(n, world, 128)[rank]
        mine, _ = oracle.detect(plane, H, ta, f_lo=lo, f_hi=hi)
        assert (mine["f"] >= lo).all() and (mine["f"] < hi).all()
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        slowest = shard.max_over_ranks(1.0 + rank, dist)
        if rank == 0:
            merged = shard.merge_records(parts, key=("k", "z", "f"))
            whole, _ = oracle.detect(plane, H, ta)
            whole = shard.merge_records([whole], key=("k", "z", "f"))
            np.save(os.path.join(out_dir, "merged.npy"), merged)
            np.save(os.path.join(out_dir, "whole.npy"), whole)
            np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_band_shards_on_two_ranks_equal_the_unsplit_plane(tmp_path):
    oracle.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged.npy")
    whole = np.load(tmp_path / "whole.npy")
    assert len(whole) > 0 and np.array_equal(merged, whole)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 2.0


@pytest.mark.parametrize("n,world,tile", [(5000, 2, 128), (128, 3, 128), (1, 1, 64),
                                          (2 ** 21, 8, 128), (1000, 7, 96)])
def test_band_bounds_cover_disjoint_aligned(n, world, tile):
    b = shard.band_bounds(n, world, tile)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == n
    for (a0, a1), (b0, b1) in zip(b, b[1:]):
        assert a1 == b0
    for lo, hi in b:
        assert lo <= hi and lo % tile == 0 and (hi == n or hi % tile == 0)
    sizes = [-(-(hi - lo) // tile) for lo, hi in b]
    assert max(sizes) - min(sizes) <= 1


def test_rank_seeds_are_distinct():
    assert len({shard.rank_seed(1, r) for r in range(64)}) == 64
    assert shard.max_over_ranks(3.5) == 3.5
