"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (no GPU).

Each rank counts its own replica of the workload; the job's time is the
slowest rank's, and its rate is the units of all ranks in that time.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                           world_size=world)
    try:
        local_ms = 10.0 * (rank + 1)  # rank 1 is the slowest
        job_ms = bench.max_over_ranks(local_ms, device="cpu")
        rate = bench.whole_job_rate(1000, 4, world, job_ms)
        out.put((rank, job_ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, rate in got:
        assert job_ms == 20.0
        assert rate == pytest.approx(1000 * 4 * 2 / 0.020)


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == 20.0
