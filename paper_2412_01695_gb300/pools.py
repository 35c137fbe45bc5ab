"""k-point pools across ranks (paper Sec. 4: k-points are split into pools, one MPI process per
GPU, no GPU-GPU communication).

The hot path has no collective: every rank owns a contiguous block of k-points and works on it
alone.  torch.distributed is used only around the timed region (a barrier, the maximum of the
ranks' times and the sum of their work), never on the data path.
"""
from __future__ import annotations


def kpool_slice(nk: int, rank: int, world: int) -> tuple:
    """Contiguous, balanced block [start, stop) of the nk k-points owned by `rank`
    (the first nk % world ranks get one extra)."""
    if world < 1 or not 0 <= rank < world or nk < 0:
        raise ValueError("bad rank/world/nk")
    base, extra = divmod(nk, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def aggregate(units: float, seconds: float):
    """(total units over ranks, max seconds over ranks, world) for the job-level rate
    total / max; a single process returns its own numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units), float(seconds), 1
    t = torch.tensor([float(units), float(seconds)], dtype=torch.float64)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item()), dist.get_world_size()
