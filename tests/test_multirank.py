"""The multi-rank path of bench.py on CPU: world size 2 over gloo.  Every rank
takes its shard of a 256 x world batch, partitioned by estimated work (weak
scaling, no exchange on the data path); the ranks meet only to take the
maximum of their step times and the sum of their updates, which is what
bench.py reports.  The shards are disjoint, cover the batch and are
balanced."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1.0 + 2.0 * rank                      # rank 1 is the slowest
    updates = 1000 * (rank + 1)
    t, u = bench.reduce_over_ranks(ms, updates, torch.device("cpu"))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    geoms, info = bench.rank_batch(16, rank, world)
    keys = [(g["body"]["kind"], tuple(g["grid"]["n"]), tuple(g["body"]["centre"])) for g in geoms]
    gathered = [None] * world
    dist.all_gather_object(gathered, keys)
    out[rank] = (gathered, info)
    dist.barrier()
    dist.destroy_process_group()


def test_world_size_two_shards_partition_the_batch():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    gathered, info = out[0]
    assert gathered == out[1][0]
    a, b = set(gathered[0]), set(gathered[1])
    assert not (a & b)
    import bench
    allk = {(g["body"]["kind"], tuple(g["grid"]["n"]), tuple(g["body"]["centre"])) for g in bench.make_batch(32)}
    assert a | b == allk
    assert info["geometries_all_ranks"] == 32 and abs(info["imbalance"]) < 0.05


def test_world_size_two_reduction():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == (3.0, 3000) and out[1] == (3.0, 3000)
