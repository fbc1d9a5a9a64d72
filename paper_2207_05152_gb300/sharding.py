"""Work split over several GPUs, one process per GPU.

Coding: the images of a batch are independent (Sec. II-B: every image is
predicted and rANS-coded on its own), so a batch is split over the ranks by
pixel count with the longest-processing-time rule, each rank encodes (and
decodes) its own images, and one all-gather of the bitstream sizes gives
every rank the offsets of the whole batch's concatenated bitstreams.  No
pixel or bitstream crosses between GPUs.

Training: data parallel.  Each rank computes the gradient of its share of
the batch with the hand-written backward pass, one all-reduce sums the
shares weighted by their batch sizes (the gradient of the whole batch's
mean loss), and every rank applies the same Adam update, so the replicas
stay identical.

The collectives go through torch.distributed (NCCL on GPUs, gloo on the
CPU); the functions take the process group as an argument and work with any
backend.  A single image is not split: its wavefront is a chain of 3H + W - 3
dependent steps, too fine for a cross-GPU exchange per step.
"""
from __future__ import annotations

from typing import Callable, Sequence


def lpt_partition(pixel_counts: Sequence[int], world_size: int):
    """Owner rank of every image: images in decreasing pixel count (ties by
    index) each go to the rank with the fewest pixels so far (ties to the
    lowest rank).  Returns (owners, per-rank pixel totals)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(pixel_counts)), key=lambda i: (-int(pixel_counts[i]), i))
    load = [0] * world_size
    owners = [0] * len(pixel_counts)
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owners[i] = r
        load[r] += int(pixel_counts[i])
    return owners, load


def shard_of(owners: Sequence[int], rank: int):
    """Indices (ascending) of the images rank `rank` codes."""
    return [i for i, o in enumerate(owners) if o == rank]


def gather_offsets(local_sizes: Sequence[int], owners: Sequence[int], rank: int, group=None):
    """Byte offsets (n + 1) of the whole batch's bitstreams laid out in image
    order, from every rank's sizes of its own images (all-gather of one
    int64 vector of n entries, zero where another rank owns the image)."""
    import torch
    import torch.distributed as dist
    n = len(owners)
    mine = shard_of(owners, rank)
    if len(local_sizes) != len(mine):
        raise ValueError("one size per image of this rank's shard")
    sizes = torch.zeros(n, dtype=torch.int64)
    for i, s in zip(mine, local_sizes):
        sizes[i] = int(s)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        backend = dist.get_backend(group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
        parts = [torch.zeros(n, dtype=torch.int64, device=dev) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, sizes.to(dev), group=group)
        total = torch.zeros(n, dtype=torch.int64)
        for r, p in enumerate(parts):
            p = p.cpu()
            for i in shard_of(owners, r):
                total[i] = p[i]
        sizes = total
    offs = [0]
    for s in sizes.tolist():
        offs.append(offs[-1] + int(s))
    return offs


def data_parallel_step(backward: Callable, apply: Callable, ctx, tgt, group=None):
    """One data-parallel training step.  backward(ctx, tgt) -> (loss, grad)
    gives the mean loss and gradient (float tensors) of this rank's batch;
    the ranks' gradients are summed with weights B_r / B (B the total batch)
    by one all-reduce, and apply(grad) takes the result.  Returns the whole
    batch's mean loss."""
    import torch
    import torch.distributed as dist
    B = int(tgt.shape[0])
    loss, grad = backward(ctx, tgt)
    grad = torch.as_tensor(grad)
    loss = torch.as_tensor(loss, dtype=grad.dtype, device=grad.device).reshape(1)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        count = torch.tensor([float(B)], dtype=grad.dtype, device=grad.device)
        dist.all_reduce(count, group=group)
        w = B / float(count.item())
        grad = grad * w
        loss = loss * w
        dist.all_reduce(grad, group=group)
        dist.all_reduce(loss, group=group)
    apply(grad)
    return float(loss.item())


class DataParallelTrainer:
    """A Trainer replica per rank: step() runs this rank's backward pass,
    averages the gradient over the ranks and applies Adam."""

    def __init__(self, trainer, group=None):
        self.trainer = trainer
        self.group = group

    def _backward(self, ctx, tgt):
        loss, grads = self.trainer.backward(ctx, tgt)
        return loss.clone(), grads

    def step(self, ctx, tgt) -> float:
        return data_parallel_step(self._backward, self.trainer.apply, ctx, tgt, self.group)
