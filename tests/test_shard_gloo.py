"""Multi-rank logic on CPU: two gloo ranks split one volume's seeds
round-robin, each runs its share (the oracle stands in for a rank's GPU
executor here, since this host has no GPU), and the gathered results equal
the single-process results exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1310_6736_b300 import shard, synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    w = synth.workload("spheres48")
    bins = oracle.bin_volume(w.volume, w.binning)
    seeds = oracle.seed_grid(w.dims, w.stride)
    mine = shard.shard_seeds(seeds, world, rank)
    oc = oracle.octant_climb(bins, 16, w.r_min, w.r_max, mine, w.max_iter, nthreads=1)
    ms = oracle.meanshift(bins, 16, w.r_min, w.r_max, mine, w.max_iter, nthreads=1)
    S = w.r_max - w.r_min + 1
    g_oc = shard.gather_round_robin(oc, len(seeds))
    g_ms = shard.gather_round_robin(ms, len(seeds), rows_per_unit=S)
    if rank == 0:
        np.savez(os.path.join(out_dir, "gathered.npz"),
                 **{f"oc_{k}": v for k, v in g_oc.items()},
                 **{f"ms_{k}": v for k, v in g_ms.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_round_robin_merge_inverts_the_deal():
    from paper_1310_6736_b300 import shard
    x = np.arange(3 * 11).reshape(11, 3)
    parts = [shard.shard_seeds(x, 4, r) for r in range(4)]
    assert np.array_equal(shard.merge_round_robin(parts, 11), x)
    items = np.arange(11 * 5 * 2).reshape(55, 2)              # 5 rows per unit
    parts = [items.reshape(11, 5, 2)[r::3].reshape(-1, 2) for r in range(3)]
    assert np.array_equal(shard.merge_round_robin(parts, 11, rows_per_unit=5), items)


def test_two_gloo_ranks_equal_one_process(tmp_path, ko):
    from paper_1310_6736_b300 import synth
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "gathered.npz")
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    seeds = ko.seed_grid(w.dims, w.stride)
    oc = ko.octant_climb(bins, 16, w.r_min, w.r_max, seeds, w.max_iter)
    ms = ko.meanshift(bins, 16, w.r_min, w.r_max, seeds, w.max_iter)
    for k, v in oc.items():
        assert np.array_equal(got[f"oc_{k}"], v), k
    for k, v in ms.items():
        assert np.array_equal(got[f"ms_{k}"], v), k


# ------------------------------------------------- dense sweep in z-slabs
def _oracle_slab_executor(ko, B, r_min, r_max):
    """A rank's executor with the oracle standing in for its GPU: the dense
    sweep of the halo'd slab, cut to the rank's own planes."""
    def run(slab, lo, hi):
        Y, s = ko.dense(slab, B, r_min, r_max, nthreads=1)
        return Y[lo:hi], s[lo:hi]
    return run


def _slab_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1310_6736_b300 import shard, synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    w = synth.workload("spheres48")
    # rank 0 bins the volume and broadcasts the bins (the exchange step)
    t = torch.from_numpy(oracle.bin_volume(w.volume, w.binning)) if rank == 0 else \
        torch.empty(w.volume.shape, dtype=torch.uint8)
    dist.broadcast(t, src=0)
    bins = t.numpy()
    z0, z1 = shard.z_slabs(bins.shape[0], world)[rank]
    local = shard.dense_slab(bins, w.r_max, z0, z1,
                             _oracle_slab_executor(oracle, 16, w.r_min, w.r_max))
    Y, s = shard.gather_slabs(local, bins.shape[0])
    if rank == 0:
        np.savez(os.path.join(out_dir, "slabs.npz"), Y=Y, s=s)
    dist.barrier()
    dist.destroy_process_group()


def test_dense_z_slabs_two_gloo_ranks_equal_one_process(tmp_path, ko):
    """Two gloo ranks sweep the two z-slabs of the spheres volume (48
    planes, r_max = 10 halo planes each side) and gather: the result equals
    the whole sweep exactly."""
    from paper_1310_6736_b300 import synth
    port = _free_port()
    mp.start_processes(_slab_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "slabs.npz")
    w = synth.workload("spheres48")
    Y, s = ko.dense(ko.bin_volume(w.volume, w.binning), 16, w.r_min, w.r_max)
    assert np.array_equal(got["s"], s)
    assert np.array_equal(got["Y"].view(np.uint64), Y.view(np.uint64))


@pytest.mark.parametrize("world", [3, 5, 30])
def test_dense_z_slabs_uneven_splits(ko, world):
    """Uneven splits, halos wider than a slab, and more ranks than planes
    (empty slabs): the merged slabs equal the whole sweep."""
    from paper_1310_6736_b300 import shard
    rng = np.random.default_rng(world)
    bins = rng.integers(0, 6, size=(23, 14, 17)).astype(np.uint8)     # 0 = not counted
    B, r_min, r_max = 5, 1, 6
    ex = _oracle_slab_executor(ko, B, r_min, r_max)
    parts = [shard.dense_slab(bins, r_max, z0, z1, ex)
             for z0, z1 in shard.z_slabs(bins.shape[0], world)]
    Y, s = shard.merge_slabs(parts, bins.shape[0])
    Yo, so = ko.dense(bins, B, r_min, r_max)
    assert np.array_equal(s, so)
    assert np.array_equal(Y.view(np.uint64), Yo.view(np.uint64))
    assert shard.z_slabs(23, world)[-1][1] == 23
    assert all(h0 <= z0 and h1 >= z1 and h1 - h0 <= z1 - z0 + 2 * r_max
               for z0, z1 in shard.z_slabs(23, world)
               for h0, h1 in [shard.halo_planes(z0, z1, 23, r_max)])
