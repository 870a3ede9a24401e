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


def test_batched_shards_cover_every_instance_once():
    for world in (1, 2, 3, 4, 8):
        got = sorted(i for r in range(world) for i in bench.shard_instances(64, r, world))
        assert got == list(range(64)), world
        sizes = [len(bench.shard_instances(64, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def _batched_worker(rank, world, port, seconds, dofs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.batched_job(seconds[rank], dofs[rank], dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_batched_job_two_ranks():
    """The sharded batch lasts as long as its slowest rank and covers the
    dofs of every rank (strong scaling: the batch is fixed)."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds, dofs = [1.5, 1.2], [33000000, 34031232]
    procs = [ctx.Process(target=_batched_worker, args=(r, 2, port, seconds, dofs, q)) for r in range(2)]
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
        assert got[r] == (1.5, 67031232)
    assert bench.batched_job(1.5, 10) == (1.5, 10)
