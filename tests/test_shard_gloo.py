"""Multi-process forms, as gloo ranks (world size 2): frequency bands of one
plane summed on separate ranks and gathered equal the unsplit result, through
the oracle on CPU ranks and through the library on GPU ranks; the job time is
the slowest rank's."""
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


def _gpu_rank_main(rank, world, port, out_dir):
    # one process per rank, each with its own CUDA context on device 0: the
    # ranks' kernels are independent launches that never wait on one another,
    # and the only exchange is the host-side gather of the records
    import torch
    from paper_1805_12258_gb300 import hs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        nt, n, H = 85, 100_000, 16
        plane = synth.noise(nt, n, seed=45)
        ta = synth.thresholds(1e-4, H, nt)
        fop = torch.from_numpy(plane).cuda()
        cands = hs.CandBuffer(1 << 20)
        with hs.Plan(nt, n, H, ta, assume_nonneg=True) as plan:
            lo, hi = shard.band_bounds(n, world, plan.tile_bins)[rank]
            plan.run_range(fop, cands, lo, hi)
            mine, count, st = cands.fetch()
            kernel = plan.kernel
        assert st == hs.HS_OK and count == len(mine) and kernel == "staged"
        assert (mine["bin"] >= lo).all() and (mine["bin"] < hi).all()
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        if rank == 0:
            np.save(os.path.join(out_dir, "merged.npy"),
                    shard.merge_records(parts, key=("k", "z", "bin")))
            np.save(os.path.join(out_dir, "sizes.npy"), np.array([len(p) for p in parts]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_band_shards_through_the_library_on_two_ranks(tmp_path):
    # each rank sums its band with hs_run_range; the gathered records equal
    # the oracle's over the whole plane (near-threshold points excepted)
    from test_gpu_parity import assert_matches_oracle

    from paper_1805_12258_gb300 import build
    build.build()
    oracle.build()
    world = 2
    mp.spawn(_gpu_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged.npy")
    sizes = np.load(tmp_path / "sizes.npy")
    plane = synth.noise(85, 100_000, seed=45)
    ta = synth.thresholds(1e-4, 16, 85)
    ref, near = oracle.detect(plane, 16, ta, threads=8)
    assert len(ref) > 0 and (sizes > 0).all()
    assert_matches_oracle(merged, ref, near)
