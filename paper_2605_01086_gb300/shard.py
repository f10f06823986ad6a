"""Batches over several GPUs: one process per GPU, streams sharded across ranks.

Every SymLen stream decodes on its own (Sec. 4.2: the symbol counts of a
stream's words locate all of its windows), so a batch splits across ranks with
no exchange on the data path: each rank builds a Plan over its own streams and
decodes them.  The one collective is in the backward pass: dL/dA_z sums over
every stream of every rank, so the per-rank FP64 gradients of the zone scales
(n_domains x 3 values) are all-reduced.

shard_streams partitions by longest-processing-time-first on a per-stream
cost, which bounds the largest rank's load by 4/3 of the optimum and by the
mean plus the largest stream.  The cost of decoding a stream is the HBM traffic
it moves, decode_cost = 4 S (float32 samples written) + 9 n_words (one 8-byte
word and one symlen byte read per SymLen word): the decode kernels run at a
fixed fraction of the memory bandwidth, so time follows bytes.
"""
from __future__ import annotations

import heapq

import numpy as np


def decode_cost(n_samples, n_words) -> np.ndarray:
    """Bytes a decode moves per stream: 4 S out + 9 n_words in (int64)."""
    S = np.asarray(n_samples, dtype=np.int64)
    W = np.asarray(n_words, dtype=np.int64)
    if S.shape != W.shape:
        raise ValueError("n_samples and n_words must have the same shape")
    return 4 * S + 9 * W


def shard_streams(costs, world_size: int, rank: int) -> np.ndarray:
    """Indices (ascending) of the streams that `rank` decodes.

    Streams in decreasing order of cost (ties: lower index first) go one by one
    to the rank with the least cost so far (ties: lower rank).  Every rank
    computes the same partition from the same costs (decode_cost of the
    batch's segments)."""
    return shard_assignment(costs, world_size)[1][rank]


def shard_assignment(costs, world_size: int):
    """(loads int64[world_size], [indices of each rank]) of the LPT partition."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    n = np.asarray(costs, dtype=np.int64)
    if n.ndim != 1 or (n < 0).any():
        raise ValueError("costs must be a 1-D array of non-negative numbers")
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
