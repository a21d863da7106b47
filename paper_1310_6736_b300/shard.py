"""Sharding of the hot path across ranks (one process per GPU).

Every unit of work is independent: a volume, a seed of the octant climb, a
(seed, r) item of mean shift.  So the path shards with no exchange step:

  * many volumes: each rank takes its own volumes (what bench.py does under
    torchrun: weak scaling, no data-path collective);
  * one volume, seed searches: the bin volume is small enough to replicate,
    and the seeds are dealt round-robin (seed i to rank i % world); results
    are gathered once at the end, back in seed order;
  * one volume, dense sweep: the centres are split into z-slabs, one per
    rank; a rank holds its slab's planes plus r_max halo planes on each
    side (clipped to the volume), so every window of its centres sees the
    voxels it sees in the whole volume, and sweeps only its own planes.
    The slabs' results are gathered in z order.

The exchange steps are the broadcast of the bin volume (one byte a voxel:
float32 binning needs the whole volume's minimum and maximum, so the ranks
share the bins, not the raw values) and the final gathers.  They go through
torch.distributed (broadcast, all_gather_object), so they work over nccl or
gloo.
"""
from __future__ import annotations

import numpy as np

__all__ = ["shard_seeds", "merge_round_robin", "gather_round_robin", "z_slabs", "halo_planes",
           "dense_slab", "gather_slabs", "gpu_slab_executor", "dense_sharded"]


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


def z_slabs(nz, world):
    """[z0, z1) of every rank: nz planes split as evenly as possible (the
    first nz % world ranks take one plane more; a rank may get none)."""
    base, extra = divmod(nz, world)
    out, z = [], 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def halo_planes(z0, z1, nz, r_max):
    """Planes [h0, h1) a rank must hold for centres [z0, z1): Ball(r_max)
    reaches r_max planes above and below; beyond the volume nothing is
    counted, so the halo stops there."""
    return max(0, z0 - r_max), min(nz, z1 + r_max)


def dense_slab(bins, r_max, z0, z1, executor):
    """One rank's share of a volume's dense sweep: the stored bin volume's
    halo'd planes go to executor(slab, lo, hi), which returns (Y, s_best)
    for the slab's planes [lo, hi) = [z0 - h0, z1 - h0).  Returns (z0, Y, s)."""
    bins = np.asarray(bins)
    h0, h1 = halo_planes(z0, z1, bins.shape[0], r_max)
    if z1 <= z0:
        ny, nx = bins.shape[1:]
        return z0, np.zeros((0, ny, nx), np.float64), np.zeros((0, ny, nx), np.uint8)
    Y, s = executor(np.ascontiguousarray(bins[h0:h1]), z0 - h0, z1 - h0)
    return z0, np.asarray(Y), np.asarray(s)


def merge_slabs(parts, nz):
    """(z0, Y, s) parts of every rank, in any order, back into whole-volume
    Y and s_best arrays (their planes must tile [0, nz))."""
    parts = sorted(parts, key=lambda p: p[0])
    Y = np.concatenate([p[1] for p in parts])
    s = np.concatenate([p[2] for p in parts])
    assert Y.shape[0] == nz and s.shape[0] == nz
    return Y, s


def gather_slabs(local, nz, group=None):
    """All-gather every rank's (z0, Y, s) and merge them in z order."""
    import torch.distributed as dist

    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    return merge_slabs(parts, nz)


def gpu_slab_executor(ctx, bins_count, params):
    """Executor for dense_slab on this rank's GPU: the slab becomes a
    volume of stored bins (KS_BIN_STORED) and the library sweeps only the
    rank's own planes (ks_dense_saliency_range)."""
    from . import ks

    def run(slab, lo, hi):
        v = ctx.create_volume(slab, {"kind": ks.KS_BIN_STORED, "bins": bins_count, "shift": 0,
                                     "lo": 0, "hi": 0})
        try:
            return ctx.dense_saliency_range(v, params, slab.shape, lo, hi)
        finally:
            ctx.release_volume(v)

    return run


def dense_sharded(ctx, volume, binning, params, group=None):
    """The dense sweep of one volume over every rank of `group`, one GPU
    each: rank 0 bins the volume and broadcasts the bins, every rank sweeps
    its z-slab with its r_max halo, and every rank returns the gathered
    whole-volume (Y_best, s_best)."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    nz, ny, nx = volume.shape
    if rank == 0:
        v = ctx.create_volume(volume, binning)
        bins = ctx.volume_bins(v, volume.shape)
        ctx.release_volume(v)
        t = torch.from_numpy(bins)
    else:
        t = torch.empty((nz, ny, nx), dtype=torch.uint8)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.broadcast(t, src=dist.get_global_rank(group, 0) if group is not None else 0,
                   group=group)
    bins = t.cpu().numpy()
    z0, z1 = z_slabs(nz, world)[rank]
    local = dense_slab(bins, params.r_max, z0, z1,
                       gpu_slab_executor(ctx, binning["bins"], params))
    return gather_slabs(local, nz, group)
