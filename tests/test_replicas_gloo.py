"""Replica (multi-GPU) host logic on CPU with two gloo ranks: disjoint shards and max-over-ranks timing."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1809_07592_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(replicas.shard(257, rank, world))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = replicas.max_over_ranks(1.5 + rank)
        out[rank] = (gathered, t, replicas.rank_base_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    g0, t0, s0 = out[0]
    g1, t1, s1 = out[1]
    assert g0 == g1
    allitems = sorted(i for part in g0 for i in part)
    assert allitems == list(range(257))  # every block exactly once
    assert t0 == t1 == 2.5  # the slowest rank's time
    assert s0 != s1


def test_shard_sizes_and_rate():
    for count in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(count, r, world) for r in range(world)]
            assert sum(len(p) for p in parts) == count
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    assert replicas.whole_job_rate(100.0, 4, 2.0) == 200.0
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)
