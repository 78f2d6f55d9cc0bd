"""Multi-GPU decomposition of the hot path: query points are independent solves, so they
shard across ranks with no collective on the data path.  Two host-side helpers ride on
torch.distributed: the step time reduced as the maximum over ranks, and an optional
gather of the per-query results (d + 1 numbers per query) onto every rank."""
from __future__ import annotations

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
