"""Host logic of runs on several GPUs (one process per GPU).

A single system's solve does not shard: every transform is global. Several
GPUs therefore step independent replicas (the benchmark) or independent
systems of an ensemble, with no collective on the data path. What crosses
ranks is host-side only: the slowest rank's time, the assignment of ensemble
systems to ranks, and a final gather of per-rank results. torch.distributed
carries it (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import heapq
import math
import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def system_cost(n: int, N: int) -> float:
    """Estimated cost of one step of a system: the 42 mesh transforms
    (n^3 log n each) plus the particle work (N taps sets)."""
    return 42.0 * n ** 3 * math.log2(max(n, 2)) / 64.0 + 30.0 * N


def lpt_shard(costs, world: int):
    """Longest-processing-time assignment of items (their costs) to `world`
    ranks: items in decreasing cost, each to the least-loaded rank. Returns
    one sorted list of item indices per rank."""
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: -costs[k]):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(v) for v in out]


def gather_to_root(obj, dist=None):
    """All ranks' objects on rank 0 (a list in rank order), None elsewhere;
    [obj] without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
