"""bench.py's multi-rank timing on two gloo ranks (CPU): every rank runs its
own replica of the workload, the job lasts as long as the slowest rank, and
the N replicas complete N load steps in that time."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.job_seconds_per_load_step(seconds[rank], dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_single_rank_time_is_the_step_time():
    assert bench.job_seconds_per_load_step(0.075) == (0.075, 0.075)


def test_two_ranks_slowest_and_job_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds = [0.30, 0.50]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = dict(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        slowest, job = got[r]
        assert slowest == pytest.approx(0.50, rel=0, abs=0)
        assert job == pytest.approx(0.25, rel=0, abs=0)
