"""k-point pools across ranks (paper Sec. 3: k-points are split into pools, one MPI process per
GPU, no GPU-GPU communication).

H|psi>, the Davidson and the Sternheimer CG have no collective: every rank owns a contiguous
block of k-points and works on it alone.  torch.distributed is used around the timed region (a
barrier, the maximum of the ranks' times and the sum of their work) and for the one exchange
the method has: the induced density (Eq. drho) is a sum over every k, so the pools' partial
grids are added by one all-reduce of the N^3 complex grid per perturbation (reduce_drho).
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


def reduce_drho(drho, group=None):
    """Sum, in place, the partial induced densities of all pools (Eq. drho: drho(r) sums over
    every k-point, so each pool holds the part of its own k-points).

    drho   complex128 tensor [N][N][N]: on entry this rank's partial grid, computed with the
           weights of the whole grid (w_k = 1/N_k of the full, unreduced k-set, not of the
           pool); on return the full sum on every rank.  A CUDA tensor with the nccl backend,
           a host tensor with gloo.
    One all-reduce of 2 N^3 float64 (the real view of the grid).  A single process (no
    process group) returns its grid unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return drho
    if drho.dtype != torch.complex128 or not drho.is_contiguous():
        raise ValueError("drho must be a contiguous complex128 tensor")
    dist.all_reduce(torch.view_as_real(drho), op=dist.ReduceOp.SUM, group=group)
    return drho
