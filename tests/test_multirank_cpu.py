"""Rank logic of bench.py's replica mode on two gloo processes (CPU only).

The sampler shards by chain: every rank runs its own replica (same data, MCMC
seed 1 + rank) and the only collective is the max over ranks of the timed
region. These tests run that logic without a GPU.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max = bench.max_over_ranks(1.5 + rank, "cpu", world)
    wl, w = bench.make_workload("lg_d2_T64", rank)
    cfg = bench.config_of("lg_d2_T64", w, 0, 8)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), t_max=t_max, seed=wl.mcmc_seed, y=wl.y,
             x0=wl.x_init, parallelism=cfg["parallelism"])
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_share_data_differ_in_seed_and_agree_on_max_time(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # every rank reports the slowest replica's time
    assert float(r[0]["t_max"]) == float(r[1]["t_max"]) == 2.5
    # independent replicas: same observations, different MCMC streams
    assert int(r[0]["seed"]) == 1 and int(r[1]["seed"]) == 2
    assert np.array_equal(r[0]["y"], r[1]["y"])
    assert str(r[0]["parallelism"]) == "replicas"


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu", 1) == 3.25
