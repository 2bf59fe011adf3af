"""Replica helpers for running on several GPUs of one node.

A single graph's FastSV solve does not shard: every iteration gathers and
hooks across the whole vertex set (the paper distributes it over a 2-D process
grid with all-to-all exchanges, Section 4.2).  On this platform each GPU runs
its own solves, and independent graphs -- a batch or a stream of requests --
are split across ranks with no collective on the data path.  The only
collectives are bookkeeping: a barrier around timed regions, a max-reduction
of step times, and gathering small results on rank 0.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_graphs(sizes, world: int) -> list[list[int]]:
    """Assign graph indices to ``world`` ranks so that the summed work
    (``sizes``, e.g. n + m per graph) is balanced: longest-processing-time
    first, ties broken by index, so every rank computes the same split."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    for r in range(world):
        out[r].sort()
    return out


def batch_work(batch) -> np.ndarray:
    """n_g + m_g for every graph of a graphgen.Batch-like object."""
    return np.diff(batch.vtx_off) + np.diff(batch.edge_off)


def max_over_ranks(value: float, dist=None) -> float:
    """Largest value over all ranks (timing rule: the job is as slow as its
    slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
