"""Sharding of independent matrix evaluations across ranks (one process per GPU).

The matrices of a batch are independent problems, so a batch is partitioned across ranks
with no collective on the data path: each rank evaluates its own shard with the library's
grouped entry point, and a gather is needed only if the caller wants every result on every
rank.  The partition balances an estimate of each matrix's cost,
    (products + squarings) * n^3,   products = s - 1 + floor(m/s),  s = ceil(sqrt(m)),
    squarings = max(0, ceil(log2 ||A||_1)),
by greedy longest-processing-time assignment (deterministic: ties go to the lower rank).
"""
from __future__ import annotations

import heapq
import math


def _ceil_sqrt(m: int) -> int:
    if m <= 1:
        return 1
    s = math.isqrt(m)
    return s if s * s == m else s + 1


def squarings(norm1: float) -> int:
    if not (norm1 > 1.0) or not math.isfinite(norm1):
        return 0
    mant, e = math.frexp(norm1)
    return e - 1 if mant == 0.5 else e


def cost(n: int, m: int, norm1: float) -> float:
    """Estimated work of exp by PS + scaling and squaring for one n x n matrix."""
    m = 30 if m <= 0 else m
    s = _ceil_sqrt(m)
    return float((s - 1 + m // s + squarings(norm1)) * n ** 3)


def partition(ns, ms, norms, world: int):
    """Assign items to `world` ranks: list of sorted index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [cost(n, m, a) for n, m, a in zip(ns, ms, norms)]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(sh) for sh in shards]


def shard_loads(ns, ms, norms, shards):
    return [sum(cost(ns[i], ms[i], norms[i]) for i in sh) for sh in shards]


def expm_local(mats, degrees, rank: int, world: int, policy=None):
    """Evaluate this rank's shard of exp(A_i) with the library (CUDA tensors).  Returns
    (indices, results) for the shard."""
    import torch

    import paper_2312_17396_gb300 as mpps
    ns = [int(a.shape[0]) for a in mats]
    norms = [float(a.abs().sum(dim=0).max()) for a in mats]
    shards = partition(ns, degrees, norms, world)
    mine = shards[rank]
    if not mine:
        return [], []
    outs = mpps.expm_grouped([mats[i] for i in mine], [degrees[i] for i in mine], policy=policy)
    torch.cuda.synchronize()
    return mine, outs


def gather_results(indices, results, count: int, group=None):
    """All ranks' (index, result) pairs -> list of `count` results on every rank (host
    tensors).  Uses torch.distributed.all_gather_object: result collection only."""
    import torch.distributed as dist
    local = [(i, r.detach().cpu()) for i, r in zip(indices, results)]
    world = dist.get_world_size(group)
    bucket = [None] * world
    dist.all_gather_object(bucket, local, group=group)
    out = [None] * count
    for part in bucket:
        for i, r in part:
            out[i] = r
    return out
