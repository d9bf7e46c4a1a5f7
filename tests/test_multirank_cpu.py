"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each rank
works on its own matrix, the job time is the maximum over ranks, whole-job
throughput counts every rank's matrix, and a batch is sharded across ranks with
no data-path collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        q.put((rank, ms, seeds))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_distinct_problems():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, seeds in out:
        assert ms == 150.0                      # the maximum over ranks
        assert seeds == [0, 1]                  # each rank its own matrix
    # whole-job value: ms per matrix = step time / matrices processed by all ranks
    assert 150.0 / 2 == 75.0


def test_shard_batch_balances_and_covers():
    flops = [float(x) for x in [9, 1, 7, 3, 5, 5, 2, 8]]
    parts = bench.shard_batch(flops, 3)
    assert sorted(k for p in parts for k in p) == list(range(len(flops)))
    loads = [sum(flops[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(flops)
    assert bench.shard_batch(flops, 1) == [sorted(range(8), key=lambda k: -flops[k])]


def test_single_rank_time_is_local():
    assert bench.max_over_ranks(12.5, None) == 12.5
