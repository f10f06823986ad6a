"""Batches over several GPUs: one process per GPU, streams sharded across ranks.

Every SymLen stream decodes on its own (Sec. 4.2: the symbol counts of a
stream's words locate all of its windows), so a batch splits across ranks with
no exchange on the data path: each rank builds a Plan over its own streams and
decodes them.  The one collective is in the backward pass: dL/dA_z sums over
every stream of every rank, so the per-rank FP64 gradients of the zone scales
(n_domains x 3 values) are all-reduced.

shard_streams partitions by longest-processing-time-first on the sample
counts (decode time is proportional to samples), which bounds the largest
rank's load by 4/3 of the optimum and by the mean plus the largest stream.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_streams(n_samples, world_size: int, rank: int) -> np.ndarray:
    """Indices (ascending) of the streams that `rank` decodes.

    Streams in decreasing order of n_samples (ties: lower index first) go one by
    one to the rank with the least samples so far (ties: lower rank).  Every
    rank computes the same partition from the same lengths."""
    return shard_assignment(n_samples, world_size)[1][rank]


def shard_assignment(n_samples, world_size: int):
    """(loads int64[world_size], [indices of each rank]) of the LPT partition."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    n = np.asarray(n_samples, dtype=np.int64)
    if n.ndim != 1 or (n < 0).any():
        raise ValueError("n_samples must be a 1-D array of non-negative counts")
    order = np.lexsort((np.arange(n.size), -n))
    heap = [(0, r) for r in range(world_size)]
    owner = np.empty(n.size, dtype=np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(n[i]), r))
    parts = [np.flatnonzero(owner == r) for r in range(world_size)]
    loads = np.array([int(n[p].sum()) for p in parts], dtype=np.int64)
    return loads, parts


def allreduce_scale_grad(grad_scale, group=None):
    """Sums the FP64 zone-scale gradients [n_domains, 3] of every rank, in place."""
    import torch
    import torch.distributed as dist

    if grad_scale.dtype != torch.float64:
        raise TypeError("grad_scale must be float64")
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(grad_scale, op=dist.ReduceOp.SUM, group=group)
    return grad_scale


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest value over all ranks (a time measured on each rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
