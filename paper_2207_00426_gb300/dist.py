"""Host logic for running the smoothers on several GPUs (one process per GPU).

Sequences are independent (each has its own prior and observations), so a
batch is sharded by sequence and every rank smooths its own shard with no
collective on the data path.  The only exchange is a sum over ranks of the
per-rank negative log-likelihood and gradient (1 + len(theta) values) when a summed
objective is wanted, and a max over ranks of timings.

shard_sequences   longest-processing-time assignment of sequences to ranks
                  (balances the total number of time steps).
shard_offsets     the offsets of one rank's shard, for the C ABI.
allreduce_sum / allreduce_max   thin wrappers over torch.distributed (any
                  backend; CPU tensors so that gloo works).
"""
import heapq

import numpy as np
import torch


def shard_sequences(lengths, world):
    """Assign sequence indices to `world` ranks, longest first, each to the
    rank with the fewest steps so far.  Returns a list of index arrays
    (ascending within a rank)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in np.argsort(-lengths, kind="stable"):
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(lengths[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_offsets(lengths, idx):
    """Offsets (len(idx) + 1) of the sequences `idx`, concatenated."""
    lengths = np.asarray(lengths, dtype=np.int64)[idx]
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    return off


def gather_rows(y, offsets, idx):
    """Rows of the sequences `idx` of a concatenated array."""
    return np.concatenate([y[offsets[i]:offsets[i + 1]] for i in idx]) if len(idx) else y[:0]


def allreduce_sum(values, group=None):
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(values, dtype=np.float64)).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


def allreduce_max(value, group=None):
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
