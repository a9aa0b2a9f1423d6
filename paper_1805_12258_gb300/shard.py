"""Host logic of the multi-GPU forms (one process per GPU).

Independent planes (beams, DM trials) shard with no exchange: each rank sums
its own planes (the paper runs separate boards on separate half planes,
Section VI-C).  One plane shards by frequency band: output bins [a, b) need
level m's inputs [a/m, b/m), all below b, so with the plane resident on every
rank a band needs nothing from any other rank; the ranks' candidate lists are
concatenated (all-gather) at the end.  The only collectives are the timing
barrier, the max over ranks of the elapsed time and, for bands, the gather of
candidates.
"""
from __future__ import annotations

import numpy as np


def band_bounds(n_bins: int, world: int, tile: int) -> list[tuple[int, int]]:
    """Split output bins [0, n_bins) into `world` contiguous bands whose
    inner edges are multiples of `tile`, balanced in tiles."""
    if n_bins < 1 or world < 1 or tile < 1:
        raise ValueError("n_bins, world and tile must be positive")
    n_tiles = -(-n_bins // tile)
    edges = [min(n_bins, (r * n_tiles // world) * tile) for r in range(world + 1)]
    edges[-1] = n_bins
    return [(edges[r], edges[r + 1]) for r in range(world)]


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own plane in the independent-planes form."""
    return int(base_seed) + 1000 * int(rank)


def merge_records(parts, key=("k", "z", "bin")) -> np.ndarray:
    """Concatenate the ranks' candidate records and sort them by (k, z, bin)."""
    parts = [p for p in parts if p is not None]
    if not parts:
        return np.zeros(0)
    r = np.concatenate(parts)
    if len(r) == 0:
        return r
    return r[np.lexsort(tuple(r[f] for f in reversed(key)))]


def max_over_ranks(value: float, dist=None) -> float:
    """The largest value over the ranks of the default process group (the
    value itself without one): the job's elapsed time is the slowest rank's."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
