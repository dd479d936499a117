"""Path-range sharding over ranks (one process per GPU).

Paths are independent and the counter-based random numbers depend only on
the global path index, so P paths split into contiguous ranges, one per
rank, reproduce the single-GPU estimate exactly up to reduction order. The
only exchange is one sum of the 3 + n_spot * n_time raw sums (LV_SUM_*
layout) across ranks; every rank then finalizes the same totals.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple


def path_range(rank: int, world: int, n_paths: int) -> Tuple[int, int]:
    """Contiguous range of global path indices owned by `rank`."""
    if not (0 <= rank < world) or n_paths < 0:
        raise ValueError("bad rank / world / n_paths")
    return n_paths * rank // world, n_paths * (rank + 1) // world


def sharded_sums(sums_fn: Callable[[int, int], "object"], n_paths: int, group=None):
    """Sum over all ranks of sums_fn(begin, end) for this rank's path range;
    sums_fn returns a torch tensor of raw sums (any device the process group
    can reduce). Ranks with an empty range contribute zeros."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    b, e = path_range(rank, world, n_paths)
    part = sums_fn(b, e) if e > b else None
    if part is None:
        ref = sums_fn(0, 1)                      # shape and device only
        part = torch.zeros_like(ref)
    part = part.clone()
    if world > 1:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def price_greeks_sharded(surface, S0, r, K, T, n_steps, n_paths, seed, stream_id: int = 0, group=None,
                         device: Optional["object"] = None):
    """Price, delta and vegas of one option over n_paths paths split across
    the ranks of `group` (NCCL for CUDA tensors): each rank runs the adjoint
    on its range, the raw sums are summed across ranks, and each rank
    finalizes them on its GPU. Returns a device tensor [3 + I*J] (LV_OUT_*)."""
    import torch

    dev = device or torch.device("cuda", torch.cuda.current_device())
    n = 3 + surface.n_spot * surface.n_time

    def run(b, e):
        out = torch.zeros(n, dtype=torch.float64, device=dev)
        surface.price_greeks_sums_device(S0, r, K, T, n_steps, b, e, seed, stream_id, out.data_ptr())
        return out

    surface.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    total = sharded_sums(run, n_paths, group)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    surface.finalize_sums_device(total.data_ptr(), n_paths, S0, out.data_ptr())
    return out
