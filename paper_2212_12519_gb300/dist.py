"""Multi-GPU arithmetic of the projector (one process per GPU).

The hot path shards naturally: LORs (or events) split into contiguous ranges
per rank, every rank holds the image, forward outputs are disjoint, and a
back projection is a sum over LORs, so the ranks' partial images add up to
the whole with one sum-allreduce of the image; an OSEM subset update needs
one such allreduce per subset.  Independent frames (the
benchmark's batches, the served OSEM frames) need no collective at all.
The local projector is passed in, so the same code runs the CUDA library on
GPUs and any other projector in tests.
"""
from __future__ import annotations

from typing import Callable, Tuple

import torch
import torch.distributed as dist


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous balanced range [start, end) of n items for this rank."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def back_allreduce(local_back: Callable[[int, int], torch.Tensor], n: int, group=None) -> torch.Tensor:
    """A^T y over all n LORs: every rank back-projects its shard with
    ``local_back(start, end)`` and one sum-allreduce adds the images."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    s, e = shard(n, rank, world)
    img = local_back(s, e)
    dist.all_reduce(img, op=dist.ReduceOp.SUM, group=group)
    return img


def fwd_gather(local_fwd: Callable[[int, int], torch.Tensor], n: int, group=None) -> torch.Tensor:
    """A x over all n LORs: disjoint shards, gathered in LOR order (only
    needed when one rank wants the whole projection)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    s, e = shard(n, rank, world)
    part = local_fwd(s, e)
    sizes = [shard(n, r, world)[1] - shard(n, r, world)[0] for r in range(world)]
    m = max(sizes)
    padded = torch.zeros((m,) + tuple(part.shape[1:]), dtype=part.dtype, device=part.device)
    padded[: part.shape[0]] = part
    out = [torch.empty_like(padded) for _ in sizes]
    dist.all_gather(out, padded, group=group)
    return torch.cat([o[:sz] for o, sz in zip(out, sizes)])


def osem_subset_allreduce(x: torch.Tensor, local_bp: Callable[[torch.Tensor], torch.Tensor],
                          update: Callable[[torch.Tensor, torch.Tensor], torch.Tensor], group=None) -> torch.Tensor:
    """One OSEM subset update with the subset's events (or LORs) sharded over
    ranks: every rank back-projects the ratio of its own events,
    ``local_bp(x)`` (forward projection, ratio and back projection are local
    per event), one sum-allreduce of the image adds the shards, and every
    rank applies the same multiplicative ``update(x, bp)``, so the replicas
    of x stay identical."""
    bp = local_bp(x)
    dist.all_reduce(bp, op=dist.ReduceOp.SUM, group=group)
    return update(x, bp)


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """Wall time of a step across ranks (the slowest rank)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
