"""The data-parallel (N > 1) path on the CPU: two `gloo` ranks, each with its
own shard, reduce their timings (max) and their work (sum) into one whole-job
rate, and their shards come from disjoint, reproducible seed streams.  A
global batch split over the ranks by contiguous pair ranges is gathered back
in global pair order (the oracle stands in for each rank's GPU outputs in
this test only)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2604_17538_b300 import scenes, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.hull_env_scene(seed=shard.shard_seed(2, rank), n_envs=3)
        units = sc.piece_pairs() + rank          # unequal work per rank
        seconds = 0.5 + rank                     # the slower rank sets the time
        total, slowest, rate = shard.job_rate(units, seconds)
        mx = shard.reduce_max([rank, -rank])
        dist.barrier()
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), pose_a=sc.pose_a, units=units,
                 total=total, slowest=slowest, rate=rate, mx=np.array(mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_work(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npz") for k in range(world)]
    units = [int(x["units"]) for x in r]
    for x in r:                                  # every rank sees the same job figures
        assert float(x["total"]) == sum(units)
        assert float(x["slowest"]) == 0.5 + (world - 1)
        assert float(x["rate"]) == pytest.approx(sum(units) / (0.5 + world - 1))
        assert list(x["mx"]) == [world - 1, 0]
    # disjoint shards, each reproducible from its rank's seed in one process
    assert not np.array_equal(r[0]["pose_a"], r[1]["pose_a"])
    from paper_2604_17538_b300 import scenes, shard
    for k in range(world):
        again = scenes.hull_env_scene(seed=shard.shard_seed(2, k), n_envs=3)
        assert np.array_equal(again.pose_a, r[k]["pose_a"])


def test_single_process_reductions_are_identities():
    from paper_2604_17538_b300 import shard
    assert shard.reduce_max([1.5, -2.0]) == [1.5, -2.0]
    assert shard.reduce_sum([3, 4]) == [3.0, 4.0]
    assert shard.job_rate(10, 2.0) == (10.0, 2.0, 5.0)
    assert shard.shard_seed(2, 0) == 2 and shard.shard_seed(2, 3) == 3002


def _gather_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2604_17538_b300 import scenes, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.hull_env_scene(seed=7, n_envs=5, workers=1)   # one global batch
        lo, hi = shard.shard_range(sc.n_pairs, rank, world)
        mine = sc.take(np.arange(lo, hi))
        ybar = np.random.default_rng(1).normal(size=(int(sc.group_offsets()[-1]), 8))
        off = sc.group_offsets()
        y = oracle.forward(mine, threads=1)                        # this rank's rows
        g, _ = oracle.gradient(mine, ybar[off[lo]:off[hi]], threads=1)
        y_all = shard.gather_rows(y)
        g_all = shard.gather_rows(g)
        if rank == 0:
            np.savez(os.path.join(out_dir, "gathered.npz"), y=y_all, g=g_all, ybar=ybar)
        else:
            assert y_all is None and g_all is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_outputs_in_pair_order(tmp_path, oracle_lib):
    import torch.multiprocessing as mp
    from paper_2604_17538_b300 import scenes, shard
    world = 2
    assert [shard.shard_range(5, k, 2) for k in range(2)] == [(0, 3), (3, 5)]
    assert [shard.shard_range(2, k, 3) for k in range(3)] == [(0, 1), (1, 2), (2, 2)]
    mp.start_processes(_gather_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = np.load(tmp_path / "gathered.npz")
    sc = scenes.hull_env_scene(seed=7, n_envs=5, workers=1)
    y = oracle_lib.forward(sc, threads=1)
    g, _ = oracle_lib.gradient(sc, r["ybar"], threads=1)
    assert r["y"].shape == y.shape and np.array_equal(r["y"], y)
    assert np.array_equal(r["g"], g)
