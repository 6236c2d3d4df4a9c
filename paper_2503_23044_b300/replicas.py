"""Data-parallel replicas of the training step (the paper distributes the
scene over GPUs and all-reduces the decoder's gradients, Sec. 3.2; here every
rank holds the whole scene and renders its own batch of views).

The views of the batch are independent until the gradient sum (the loss is a
sum of per-view terms, Eq. 8-9, and pgs_backward accumulates), so the one
exchange of a data-parallel step is a sum over ranks of the anchor and decoder
gradients: one all-reduce of a single flattened buffer per step, in the
process group's backend (NCCL between GPUs, gloo on CPU).  No collective sits
on the render/backward path itself; the benchmark's timed step stays a
single-GPU step and does not call this.
"""
from __future__ import annotations

from typing import Dict, Optional

import torch
import torch.distributed as dist


def allreduce_param_grads(param_grads: Dict[str, torch.Tensor], group: Optional[dist.ProcessGroup] = None,
                          average: bool = False) -> None:
    """Sum (or average) the gradient tensors over the ranks of ``group``, in
    place, with one all-reduce of a flattened copy (names in sorted order so
    every rank packs the same layout).  Tensors must have the same shapes and
    dtype on every rank."""
    names = sorted(param_grads)
    if not names:
        return
    flat = torch.cat([param_grads[n].reshape(-1) for n in names])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    if average:
        flat /= dist.get_world_size(group)
    off = 0
    for n in names:
        t = param_grads[n]
        k = t.numel()
        t.copy_(flat[off:off + k].view_as(t))
        off += k
