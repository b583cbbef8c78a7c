"""Placement of independent simulations on the ranks of a job, one GPU each.

The batched form's members are independent problems, so a multi-GPU job
shards them by member and needs no collective on the data path: every rank
computes the same placement from the members' sizes alone and advances its
own share as one batch.  The placement is the longest-processing-time-first
greedy rule (Graham): members in decreasing order of cost, each to the rank
with the least load so far, so that the slowest rank carries at most 4/3 of
the optimum.  The cost of a member is the bytes its step moves: three line
sweeps, each reading and writing the field once.
"""
from typing import List, Sequence


def member_cost(nx: int, ny: int, nz: int, n_sub: int, elem_bytes: int = 8) -> int:
    """Bytes one step of a member moves through its three sweeps."""
    return 3 * 2 * nx * ny * nz * n_sub * elem_bytes


def lpt_partition(costs: Sequence[float], n_ranks: int) -> List[List[int]]:
    """Member indices of each rank (each list in increasing order).  Ties
    are broken by member index and by rank, so every rank computes the same
    placement."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * n_ranks
    parts: List[List[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def problems_for_rank(problems, rank: int, world: int):
    """The share of `problems` (objects with nx, ny, nz, n_sub and
    precision) that rank `rank` of `world` advances."""
    costs = [member_cost(p.nx, p.ny, p.nz, p.n_sub, 8 if p.precision == 64 else 4)
             for p in problems]
    return [problems[i] for i in lpt_partition(costs, world)[rank]]
