"""The benchmark's multi-rank plumbing on CPU: world size 2 over gloo.

The workload does not shard (replicas only), so the only cross-rank work is
the host-side barrier and the max of the ranks' times."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist, r, w = bench.dist_init(world)
    bench.barrier(dist)
    worst = bench.max_over_ranks(dist, 1.0 + rank)
    q.put((r, w, worst))
    dist.destroy_process_group()


def test_two_ranks_barrier_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2, 2.0), (1, 2, 2.0)]


def test_single_rank_needs_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    import bench
    dist, r, w = bench.dist_init(1)
    assert dist is None and (r, w) == (0, 1)
    assert bench.max_over_ranks(None, 3.5) == 3.5
