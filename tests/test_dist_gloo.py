"""The benchmark's multi-rank bookkeeping (max of the timed region over ranks,
sum of per-rank rates for independent replicas) on two CPU ranks with gloo."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total_ms, value = bench.aggregate_ranks(10.0 + rank, 100.0 * (rank + 1), device="cpu")
    srcs = bench.replica_sources(list(range(64)), rank, world)
    q.put((rank, total_ms, value, srcs))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, value, srcs in res:
        assert total_ms == 11.0  # slowest rank's timed region
        assert value == 300.0    # replicas: the job's rate is the sum of the ranks' rates
        assert srcs == list(range(64))  # every replica runs the full 64-source workload
