"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each solving its own
replica, aggregate to units of all ranks over the max-over-ranks time."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_total = [300.0, 500.0][rank]
    units = [4e6 * 10, 4e6 * 10][rank]
    value, ms_per_step = bench.aggregate(ms_total, units, 10, dist, torch.device("cpu"))
    out.put((rank, value, ms_per_step))
    dist.destroy_process_group()


def test_two_rank_aggregate_uses_max_time_and_total_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert value == pytest.approx(8e7 / 0.5)
        assert ms == pytest.approx(50.0)


def test_single_process_aggregate():
    import bench
    value, ms = bench.aggregate(200.0, 1e6, 4, None, None)
    assert value == pytest.approx(1e6 / 0.2) and ms == pytest.approx(50.0)
