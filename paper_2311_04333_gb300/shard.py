"""Sharding of batched and serving work across GPUs by graph.

Independent graphs are the one unit of this path that splits across GPUs
with no exchange on the data path: each rank runs dsg_run_batch on its own
contiguous range of the batch, and only the small per-graph results are
gathered afterwards (torch.distributed all_gather_object, over NCCL or gloo).
A single graph is not split (its iterations need a global order of all
vertices), so single-graph work runs as independent replicas.

The split balances the work per rank: graph g costs 2 m_g + n_g (the arcs
its edge scan reads plus its vertices), and rank r takes the graphs whose
cumulative cost starts in [r W / N, (r + 1) W / N) for total cost W over N
ranks, so every rank's share is within one graph's cost of W / N.
"""
from __future__ import annotations

import numpy as np


def graph_cost(n: int, m: int) -> int:
    """Work units of one graph: 2m arcs scanned plus n vertices sorted."""
    return 2 * int(m) + int(n)


def graph_ranges(costs, world_size: int) -> list[tuple[int, int]]:
    """Contiguous graph ranges [lo, hi), one per rank, in rank order, that
    cover all graphs once and split the total cost evenly (each share is
    within max(costs) of total / world_size)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    c = np.asarray(costs, dtype=np.int64)
    if c.size and int(c.min()) < 0:
        raise ValueError("costs must be non-negative")
    start = np.concatenate([[0], np.cumsum(c)])[:-1] if c.size else np.zeros(0, np.int64)
    total = int(c.sum()) if c.size else 0
    bounds = [0]
    for r in range(1, world_size):
        # first graph whose cumulative start reaches r * total / world_size
        # (integer comparison: start * N >= r * total)
        idx = int(np.searchsorted(start * world_size, r * total, side="left"))
        bounds.append(max(idx, bounds[-1]))
    bounds.append(int(c.size))
    return [(bounds[r], bounds[r + 1]) for r in range(world_size)]


def my_range(costs, rank: int, world_size: int) -> tuple[int, int]:
    return graph_ranges(costs, world_size)[rank]


def gather_rows(local_rows: np.ndarray, world_size: int) -> np.ndarray:
    """Concatenate every rank's per-graph result rows in rank order (all ranks
    receive the whole array).  With one rank it returns the rows unchanged."""
    local_rows = np.asarray(local_rows)
    if world_size == 1:
        return local_rows
    import torch.distributed as dist
    parts = [None] * world_size
    dist.all_gather_object(parts, local_rows)
    return np.concatenate([np.asarray(p).reshape((-1,) + local_rows.shape[1:]) for p in parts], axis=0)
