"""Multi-rank host logic on CPU with the gloo backend (world size 2).

Columns shard across ranks without data exchange: every rank derives the
same LPT plan, the shares are disjoint and cover every column, the load is
balanced, and the timing reduces to the slowest rank and the total rate.
A rank that fails before the reduction is reported by the launcher.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1109_6885_gb300 import shard


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_plan_columns_lpt():
    costs = [10, 9, 8, 7, 6, 5, 4, 3, 2, 1]
    plan = shard.plan_columns(costs, 3)
    flat = sorted(i for p in plan for i in p)
    assert flat == list(range(10))
    loads = [sum(costs[i] for i in p) for p in plan]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.plan_columns([], 2) == [[], []]
    assert shard.plan_columns([5], 4)[0] == [0] or any(p == [0] for p in shard.plan_columns([5], 4))


def test_column_cost_is_the_algorithmic_bytes():
    c = shard.column_cost(8, 1_000_000, 170_000, 20, 100_000_000, 1_000_000)
    assert c > 250_000_000 + 252_500_000


def _worker(rank, world, port, costs, times, fail_rank, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("rank failed before the reduction")
        plan = shard.plan_columns(costs, world)
        mine = plan[rank]
        units = sum(costs[i] for i in mine)
        slowest = shard.max_over_ranks(times[rank])
        rate = shard.aggregate_rate(units, times[rank])
        out.put((rank, mine, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [300, 200, 100, 250, 50, 75]
    times = [1.5, 2.0]
    mp.start_processes(_worker, args=(2, free_port(), costs, times, -1, q), nprocs=2, join=True,
                       start_method="spawn")
    res = sorted(q.get() for _ in range(2))
    shares = [r[1] for r in res]
    assert sorted(i for s in shares for i in s) == list(range(len(costs)))
    assert not set(shares[0]) & set(shares[1])
    for _, _, slowest, rate in res:
        assert slowest == 2.0
        assert rate == pytest.approx(sum(costs) / 2.0)


def test_failed_rank_is_reported():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with pytest.raises(Exception):
        mp.start_processes(_worker, args=(2, free_port(), [1, 2], [1.0, 1.0], 1, q), nprocs=2,
                           join=True, start_method="spawn")
