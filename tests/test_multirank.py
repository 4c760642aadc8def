"""Replica sharding across ranks (no data-path collective), on CPU with gloo.

Viewpoints are independent (no exchange between viewpoint PCs in the paper's
system), so each rank densifies its own views; the only collectives are the
benchmark's barrier and the max over ranks of the timed duration.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    # rank r's steps take (r + 1) ms each: the job time is the slowest rank's
    steps = [float(rank + 1)] * 5

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, total_ms = bench.job_throughput(steps, 8, world, reduce_max)
    dist.barrier()
    q.put((rank, gathered, value, total_ms))
    dist.destroy_process_group()


def test_two_ranks_shard_views_and_take_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, value, total_ms in out:
        s0, s1 = set(gathered[0]), set(gathered[1])
        assert len(s0) == 4 and not (s0 & s1)          # disjoint views per rank
        assert total_ms == pytest.approx(10.0)          # slowest rank: 5 steps x 2 ms
        assert value == pytest.approx(2 * 8 * 5 / 0.010)  # all frames over the slowest time


def test_single_rank_is_identity():
    import bench
    value, total = bench.job_throughput([1.0, 1.0], 4, 1, lambda x: x)
    assert total == 2.0 and value == pytest.approx(4000.0)
