"""The multi-GPU path of bench.py on CPU with gloo (world size 2): every rank
solves its own batch (disjoint seeds), and the job time is the slowest rank's
while the work is summed - no data-path collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        updates = 1000 * (rank + 1)
        t, u = bench.reduce_over_ranks(ms, updates, world, "cpu")
        seeds = list(range(bench.rank_seed0(rank, 4), bench.rank_seed0(rank, 4) + 4))
        obj = [None] * world
        dist.all_gather_object(obj, seeds)
        out[rank] = (t, u, obj)
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_disjoint_batches():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, u, seeds = res[rank]
        assert t == 150.0 and u == 3000
        assert not set(seeds[0]) & set(seeds[1])
