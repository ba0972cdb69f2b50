"""The multi-rank benchmark path on CPU: two gloo ranks, replicas only (no data exchanged)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 100 ms for 5 steps
        T, v = bench.aggregate_ms((rank + 1) * 100.0, 5, world, dist, "cpu")
        out[rank] = (T, v, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_divide_by_all_steps():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        T, v, seed = out[r]
        assert T == 200.0                 # the slowest rank
        assert v == 200.0 / (5 * world)   # whole-job ms per step
    assert out[0][2] != out[1][2]         # independent problems


def test_single_rank_needs_no_process_group():
    T, v = bench.aggregate_ms(123.0, 3, 1)
    assert T == 123.0 and v == 41.0
