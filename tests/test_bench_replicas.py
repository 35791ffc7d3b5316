"""The replica aggregation of bench.py (max over ranks, whole-job throughput),
exercised with two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [120.0, 150.0][rank]            # rank 1 is the slow one
    t, value = bench.job_time_and_value(elapsed, steps=10, device="cpu")
    q.put((rank, t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_aggregate_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in out:
        assert t == 150.0                       # max over ranks
        assert abs(value - 2 * 10 / 0.150) < 1e-9  # world_size * steps / slowest time


def test_single_process_is_unchanged():
    import bench
    t, value = bench.job_time_and_value(200.0, steps=4, device="cpu")
    assert t == 200.0 and abs(value - 20.0) < 1e-12
