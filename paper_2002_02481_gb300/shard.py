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
                         device: Optional["object"] = None, sums=None, out=None):
    """Price, delta and vegas of one option over n_paths paths split across
    the ranks of `group` (NCCL for CUDA tensors): each rank runs the adjoint
    on its range into raw sums, the sums are summed across ranks (the one
    exchange), and each rank finalizes the totals on its device. Returns
    `out` (or a new tensor) [3 + I*J] in the LV_OUT_* layout.

    `sums` and `out` may be passed preallocated ([3 + I*J] float64 on
    `device`) so that repeated calls allocate nothing. `surface` is an
    lv.Surface, or anything with the same price_greeks_sums_device /
    finalize_sums_device methods writing through data pointers."""
    import torch
    import torch.distributed as dist

    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    n = 3 + surface.n_spot * surface.n_time
    if dev.type == "cuda":
        surface.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    b, e = path_range(rank, world, n_paths)
    part = sums if sums is not None else torch.empty(n, dtype=torch.float64, device=dev)
    if e > b:
        surface.price_greeks_sums_device(S0, r, K, T, n_steps, b, e, seed, stream_id, part.data_ptr())
    else:
        part.zero_()
    if world > 1:
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    res = out if out is not None else torch.empty(n, dtype=torch.float64, device=dev)
    surface.finalize_sums_device(part.data_ptr(), n_paths, S0, res.data_ptr())
    return res
