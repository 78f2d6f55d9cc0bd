"""Multi-GPU decomposition of the hot path: query points and batch instances are
independent solves, so they shard across ranks with no collective on the data path.
Query points of one problem split into equal contiguous blocks (query_shard); the uneven
instances of a batch split by their estimated cost (cost_shard: largest first onto the
least loaded rank).  Host-side helpers ride on torch.distributed: the step time reduced as
the maximum over ranks, and gathers of the per-query or per-instance results."""
from __future__ import annotations

import math

import numpy as np


def query_shard(q_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of query indices owned by `rank`: (first, count); the first
    q_total % world ranks hold one extra query."""
    if world < 1 or not 0 <= rank < world or q_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(q_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device="cpu") -> float:
    """All-reduce MAX of one float (the whole-job step time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_queries(local: np.ndarray, q_total: int, device="cpu") -> np.ndarray:
    """Concatenate every rank's rows (its query block, in rank order) into [q_total, ...]."""
    import torch
    import torch.distributed as dist
    local = np.ascontiguousarray(local, dtype=np.float64)
    if not dist.is_available() or not dist.is_initialized():
        return local
    world = dist.get_world_size()
    counts = [query_shard(q_total, r, world)[1] for r in range(world)]
    width = int(np.prod(local.shape[1:])) if local.ndim > 1 else 1
    mx = max(counts)
    buf = torch.zeros(mx, width, dtype=torch.float64, device=device)
    buf[: local.shape[0]] = torch.from_numpy(local.reshape(local.shape[0], width)).to(device)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    rows = [p[:c].cpu().numpy() for p, c in zip(parts, counts)]
    out = np.concatenate(rows, axis=0)
    return out.reshape((q_total,) + local.shape[1:])


def instance_cost(w) -> float:
    """Estimated time of one instance, in seconds: N levels of 2 + sqrt(kappa) passes over
    its rows (the row step and the moments, then CG passes growing like the square root of
    the regression's condition number kappa, estimated from the Marchenko-Pastur edges of
    the cloud's covariance and the ridge), each pass a fixed launch latency of 25 us plus
    its rows at 6.5 TB/s.  The plan's branch scheduler uses the same model."""
    from .autotune import kappa_estimate
    nbytes = float(w.Q) * w.M * w.d * (4.0 if w.precision == "fp32" else 8.0)
    return w.N * (2.0 + math.sqrt(kappa_estimate(w))) * (25e-6 + nbytes / 6.5e12)


def cost_shard(instances, world: int) -> list[list[int]]:
    """Instance indices per rank: largest estimated cost first, each onto the rank with the
    least total so far (ties: the lower rank; equal costs keep instance order), every list
    in increasing index order.  Deterministic, so every rank computes the same split."""
    if world < 1:
        raise ValueError("bad shard arguments")
    costs = [instance_cost(w) for w in instances]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_instances(local: dict, n_total: int) -> list:
    """Every rank's {instance index: result} merged onto every rank, as a list in instance
    order (results of uneven size, e.g. (u0, grad u) with each instance's own d)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        merged = dict(local)
    else:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
        merged = {}
        for part in parts:
            merged.update(part)
    if sorted(merged) != list(range(n_total)):
        raise ValueError("the shards do not cover every instance exactly once")
    return [merged[i] for i in range(n_total)]
