"""Data-parallel sharding of pixels across ranks (one process per GPU).

Pixels are independent (the method inverts each on its own; the paper proposes
one GPU per scanline range), and every random draw is keyed by the global
pixel id, so a rank that inverts pixel ids [start, start + count) produces
exactly the results a single process would for those ids.  No collective
touches the data path; only timings are reduced.
"""
from __future__ import annotations


def weak_range(rank: int, world: int, npix_per_rank: int):
    """Weak scaling: rank r owns ids [r * n, (r + 1) * n)."""
    if not 0 <= rank < world or npix_per_rank < 0:
        raise ValueError("bad rank/world/npix")
    return rank * npix_per_rank, npix_per_rank


def strong_range(rank: int, world: int, npix_total: int):
    """Strong scaling: a fixed map split into contiguous, nearly equal ranges."""
    if not 0 <= rank < world or npix_total < 0:
        raise ValueError("bad rank/world/npix")
    base, extra = divmod(npix_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None) -> float:
    """Max of a per-rank scalar (the step time) over the process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
