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
