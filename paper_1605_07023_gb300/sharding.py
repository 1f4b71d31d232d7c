"""How the gridding path shards over several GPUs: weak scaling over independent problems.

Gridding of one observation onto one grid has no cheap split: two ranks
sharing a grid would need a reduction of the whole grid. The workloads do
contain independent problems, though: separate observations, and separate
(channel, w-plane) grids in a batch (Sec. 5 grids each w-slice as its own
kernel instance). Ranks therefore take whole problems, with no collective on
the data path. The only collectives are the benchmark's timing reductions
(max over ranks) and its totals (sum over ranks).
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the independent observation that `rank` grids (rank 0 keeps the base seed)."""
    return base_seed + 1_000_003 * rank


def partition_by_work(work: list[int], world: int) -> list[list[int]]:
    """Assign independent problems to ranks, balancing the summed work.

    Longest-processing-time-first greedy assignment. Returns one list of
    problem indices per rank, each sorted ascending. Deterministic: ties go to
    the lowest rank and the lowest index.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(work)), key=lambda k: (-work[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += work[i]
    return [sorted(x) for x in out]


def my_share(work: list[int], rank: int, world: int) -> list[int]:
    return partition_by_work(work, world)[rank]


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(x: float, device=None) -> float:
    """Max over ranks (the slowest rank sets the time)."""
    return _reduce(x, "max", device)


def reduce_sum(x: float, device=None) -> float:
    """Sum over ranks (whole-job totals)."""
    return _reduce(x, "sum", device)
