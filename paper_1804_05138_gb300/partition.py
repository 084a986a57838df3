"""Share of a batch of independent factorizations per GPU (host logic, no compute).

The matrices of a batch are independent problems, so a batch shards across ranks with no
exchange on the data path: rank r factors its own subset, and the only collective is the
optional gather of results.  The subsets come from longest-processing-time-first (LPT) list
scheduling (Graham 1969) on each matrix's counted flops: matrices in decreasing cost, each given
to the rank with the least total so far (ties to the lowest rank), which keeps every rank's total
within the largest single cost of every other's.
"""
from __future__ import annotations


def lpt_partition(costs, world: int) -> list[list[int]]:
    """Indices of `costs` per rank (each list in decreasing cost); every index appears once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += float(costs[i])
    return parts


def rank_loads(costs, parts) -> list[float]:
    return [sum(float(costs[i]) for i in part) for part in parts]
