"""Multi-GPU partitioning of the batched precoder.

Instances are independent, so a batch is split into contiguous ranges, one per
rank, and the forward path needs no collective at all.  Training averages the
loss and the 2T parameter gradients over the whole batch: every rank reduces
its shard on its GPU (fixed-order FP64 mean), then one all-reduce of 2T + 2
numbers, weighted by shard size, gives the global mean.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(B: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of the instances rank `rank` owns: contiguous, sizes differ by <= 1."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_mean(loss: torch.Tensor, dstep: torch.Tensor, dlam: torch.Tensor | None,
                   n_local: int, group=None):
    """Global batch mean of per-shard means: sum_r n_r x_r / sum_r n_r, in FP64.

    loss: [1] or scalar, dstep / dlam: [T]; returns the same quantities averaged over
    all ranks (in place on float copies)."""
    parts = [loss.reshape(1).double() * n_local, dstep.double() * n_local]
    if dlam is not None:
        parts.append(dlam.double() * n_local)
    parts.append(torch.tensor([float(n_local)], dtype=torch.float64, device=dstep.device))
    buf = torch.cat(parts)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    n = buf[-1]
    T = dstep.numel()
    out_loss = (buf[0] / n).to(loss.dtype)
    out_dstep = (buf[1:1 + T] / n).to(dstep.dtype)
    out_dlam = (buf[1 + T:1 + 2 * T] / n).to(dlam.dtype) if dlam is not None else None
    return out_loss, out_dstep, out_dlam
