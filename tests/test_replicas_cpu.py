"""The N > 1 path of bench.py (replicas only: one process per GPU, no
data-path collective) exercised with the gloo backend at world size 2 on
the CPU: the barrier, the max over ranks of the timed region, the whole-job
value and the per-rank chain streams."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        ms = 100.0 + 50.0 * rank  # the ranks' own timed regions
        ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
        value = bench.replica_value(world, 10, ms_max)
        # each replica's chains come from its own Philox stream (stream id = rank)
        s = oracle.chain_init(36, 8, "exchange", 2, rank)
        gathered = [torch.zeros(8 * 36, dtype=torch.int8) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(s.reshape(-1).copy()))
        out.put((rank, ms_max, value, [g.numpy() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_replicas_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ms_max, value, gathered in res:
        assert ms_max == 150.0  # the slowest rank sets the time on every rank
        assert value == pytest.approx(2 * 10 / 0.150)
    g = res[0][3]
    assert not np.array_equal(g[0], g[1])  # independent replicas
    for r in range(world):
        np.testing.assert_array_equal(g[r], oracle.chain_init(36, 8, "exchange", 2, r).reshape(-1))
        assert (g[r].reshape(8, 36).astype(int).sum(axis=1) == 0).all()
