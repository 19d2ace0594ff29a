"""The weak-scaling path of the benchmark on CPU: two gloo ranks (the GPU
runs use one process per GPU over NCCL the same way).  Each rank runs an
independent problem (its own seed); the whole-job figure is the summed work
over the slowest rank's time; no collective touches the data path."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench.dist_env()
        red = bench.RankReduce(dist, "cpu")
        ms = 10.0 + 5.0 * rank            # rank 1 is the slower one
        units = 1000.0 * (rank + 1)
        q.put((r, ws, bench.rank_seed(r), red.max(ms), red.sum(units), red.rate(units, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert [g[2] for g in got] == [1, 2]            # independent problems
    for _, _, _, mx, sm, rate in got:
        assert mx == 15.0 and sm == 3000.0           # slowest rank, summed work
        assert rate == pytest.approx(3000.0 / 15e-3)


def test_single_rank_is_identity():
    red = bench.RankReduce(None)
    assert red.max(3.0) == 3.0 and red.sum(4.0) == 4.0 and red.rate(10.0, 2.0) == pytest.approx(5000.0)
