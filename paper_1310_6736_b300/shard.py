"""Sharding of the hot path across ranks (one process per GPU).

Every unit of work is independent: a volume, a seed of the octant climb, a
(seed, r) item of mean shift.  So the path shards with no exchange step:

  * many volumes: each rank takes its own volumes (what bench.py does under
    torchrun: weak scaling, no data-path collective);
  * one volume: the bin volume is small enough to replicate, and the seeds
    are dealt round-robin (seed i to rank i % world); results are gathered
    once at the end, back in seed order.

Only the final gather is a collective.  It goes through
torch.distributed.all_gather_object, so it works over nccl or gloo.
"""
from __future__ import annotations

import numpy as np

__all__ = ["shard_seeds", "merge_round_robin", "gather_round_robin"]


def shard_seeds(seeds, world, rank):
    """Seeds of `rank`: rows rank, rank + world, rank + 2*world, ..."""
    seeds = np.asarray(seeds).reshape(-1, 3)
    return seeds[rank::world]


def merge_round_robin(parts, n_units, rows_per_unit=1):
    """Inverse of the round-robin deal.  parts[k] holds, for the units k,
    k + world, ..., `rows_per_unit` consecutive rows each (1 for octant
    seeds, S for mean-shift items)."""
    world = len(parts)
    first = next(p for p in parts if p is not None and len(p))
    out = np.empty((n_units * rows_per_unit,) + first.shape[1:], dtype=first.dtype)
    view = out.reshape((n_units, rows_per_unit) + first.shape[1:])
    for k, p in enumerate(parts):
        if p is None or not len(p):
            continue
        view[k::world] = np.asarray(p).reshape((-1, rows_per_unit) + first.shape[1:])
    return out


def gather_round_robin(local, n_units, rows_per_unit=1, group=None):
    """All-gather each rank's rows (an array, or a dict of arrays with the
    same leading layout) and merge them back into unit order on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    if isinstance(local, dict):
        return {k: merge_round_robin([p[k] for p in parts], n_units, rows_per_unit)
                for k in local}
    return merge_round_robin(parts, n_units, rows_per_unit)
