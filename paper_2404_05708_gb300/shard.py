"""Sharding independent pairs over ranks (one process per GPU).

The pairs of a batch or matrix are independent, so N GPUs take disjoint
subsets with no collective on the data path; only the timing (max over
ranks) and, when wanted, the results are combined afterwards.  The split is
longest-processing-time greedy on the cell count n*m, computed identically
by every rank from the curve lengths.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_assign(costs: np.ndarray, world: int) -> np.ndarray:
    """Rank of every item: costliest first, each to the least-loaded rank."""
    costs = np.asarray(costs, dtype=np.float64)
    owner = np.empty(costs.shape[0], dtype=np.int64)
    heap = [(0.0, r) for r in range(world)]
    for i in np.argsort(-costs, kind="stable"):
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + costs[i], r))
    return owner


def shard_pairs(lengths: np.ndarray, pairs: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Indices of the pairs this rank computes (sorted)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    pairs = np.asarray(pairs).reshape(-1, 2)
    if world == 1:
        return np.arange(pairs.shape[0])
    owner = lpt_assign(lengths[pairs[:, 0]] * lengths[pairs[:, 1]], world)
    return np.nonzero(owner == rank)[0]


def gather(values: np.ndarray, index: np.ndarray, total: int, group=None) -> np.ndarray:
    """Assemble every rank's (index, value) shard into one array on all ranks."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts_i = [None] * world
    parts_v = [None] * world
    dist.all_gather_object(parts_i, np.asarray(index), group=group)
    dist.all_gather_object(parts_v, np.asarray(values), group=group)
    out = np.zeros(total, dtype=np.asarray(values).dtype)
    for i, v in zip(parts_i, parts_v):
        out[i] = v
    del torch
    return out


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
