"""The N > 1 host path of the bench, as two gloo ranks on CPU.

The large-factorization workload shards by problem: every rank factors its
own matrices (disjoint generator seeds) and the only cross-rank exchange is
the maximum of the step times, so the reported rate is the slowest rank's
(weak scaling, no data-path collective)."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, _ = bench.env_rank()
        t = bench.max_over_ranks(0.25 + 0.5 * r, torch.device("cpu"), w)
        seeds = [bench.input_seed(r, i) for i in range(len(bench.KAPPAS))]
        q.put((r, w, t, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_is_the_slowest_and_problems_are_disjoint():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == pytest.approx(0.75) for r in res)          # max over ranks, seen by every rank
    assert set(res[0][3]).isdisjoint(res[1][3])                    # each rank its own problems
    assert all(p.exitcode == 0 for p in procs)
