"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1) run the
cross-rank aggregation the bench uses under torchrun, each with its own
step time; every rank must see the slowest time, and the whole-job
throughput counts both ranks' units over that time (weak scaling: the
path is replicated, no data moves between ranks)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        value = bench.job_throughput(128, slowest, world)
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.25, 0.40]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == 0.40
        assert value == pytest.approx(2 * 128 / 0.40)


def test_single_process_passthrough():
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_throughput(10, 2.0, 1) == 5.0
