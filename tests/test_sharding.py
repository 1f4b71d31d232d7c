"""Multi-rank host logic on CPU: gloo, world size 2 (no GPU)."""
import os
import socket

import pytest

from paper_1605_07023_gb300 import sharding


def test_partition_balances_and_covers():
    work = [1000, 10, 500, 499, 3, 3, 7000, 1]
    parts = sharding.partition_by_work(work, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(work)))
    loads = [sum(work[i] for i in p) for p in parts]
    assert max(loads) == 7000                  # the largest item alone bounds the makespan
    assert sharding.partition_by_work(work, 3) == parts     # deterministic
    assert sharding.partition_by_work(work, 1) == [list(range(len(work)))]
    with pytest.raises(ValueError):
        sharding.partition_by_work(work, 0)


def test_rank_seeds_are_distinct():
    seeds = {sharding.rank_seed(0, r) for r in range(8)}
    assert len(seeds) == 8 and sharding.rank_seed(0, 0) == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = sharding.reduce_max(10.0 + rank)
        sm = sharding.reduce_sum(1.5 * (rank + 1))
        share = sharding.my_share([5, 4, 3, 2, 1, 1], rank, world)
        q.put((rank, mx, sm, share))
    finally:
        dist.destroy_process_group()


def test_reductions_and_shares_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [4.5, 4.5]
    shares = [r[3] for r in res]
    assert sorted(shares[0] + shares[1]) == list(range(6))
    assert abs(sum([5, 4, 3, 2, 1, 1][i] for i in shares[0]) - sum([5, 4, 3, 2, 1, 1][i] for i in shares[1])) <= 1


def test_single_process_reductions_are_identity():
    assert sharding.reduce_max(3.0) == 3.0
    assert sharding.reduce_sum(3.0) == 3.0
