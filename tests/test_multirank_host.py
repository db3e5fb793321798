"""Host logic of bench.py on several ranks (no GPU): world_size 2 over gloo.

Under torchrun every rank runs its own replica (or its own share of a
many-instance workload); the job's time is its slowest rank's, taken with an
all-reduce MAX, and the reported value counts the units of all ranks.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5])
        mine = bench.shard(13, rank, ws)
        shards = [None] * ws
        dist.all_gather_object(shards, mine)
        q.put((rank, got, shards))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_timings_and_share_instances():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, shards in results:
        assert got == [2.0, 10.0, 0.5]  # every rank sees the slowest rank's times
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(13))  # each instance exactly once
        assert abs(len(shards[0]) - len(shards[1])) <= 1


def test_single_rank_helpers():
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.whole_job_rate(5.0, 2, 0.5) == 20.0
