"""Multi-rank logic of bench.py, run as two gloo ranks on the CPU.

Each rank steps its own instance (weak scaling, no collective on the data
path); the only exchange is the timing: the job's time is the slowest rank's
and the value counts every rank's grains.
"""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seconds = bench.max_over_ranks(1.0 + 0.5 * rank, "cpu")
        out.put((rank, seconds, bench.weak_value(world, 1000, seconds)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seconds, value in res:
        assert seconds == pytest.approx(1.5)
        assert value == pytest.approx(2 * 1000 / 1.5)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.weak_value(1, 300, 1.5) == pytest.approx(200.0)
