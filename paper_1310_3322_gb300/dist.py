"""Data-parallel sharding of the HMM hot path across ranks (one GPU each).

(sequence, model) pairs are independent (the paper runs one HMM per action in
parallel, Sec. 3 item 3), so recognition shards sequences across ranks with
no exchange at all; learning adds one sum of the K*(N + N*N + N*M) expected
counts per step, which is the only collective. The partition is a
length-balanced greedy split (longest sequence first onto the least-loaded
rank), deterministic for a given batch and world size.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_sequences(lengths, world: int, rank: int) -> np.ndarray:
    """Indices of the sequences rank `rank` owns (sorted ascending).

    Greedy longest-processing-time partition over sum_t 1 work units: every
    sequence goes to exactly one rank, and the heaviest rank carries at most
    the lightest rank's load plus one sequence.
    """
    lengths = np.asarray(lengths, np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    order = np.argsort(-lengths, kind="stable")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(lengths.size, np.int64)
    for s in order:
        load, r = heapq.heappop(heap)
        owner[s] = r
        heapq.heappush(heap, (load + int(lengths[s]), r))
    return np.nonzero(owner == rank)[0]


def subset(symbols, offsets, lengths, idx):
    """Packs the sequences `idx` into a new (symbols, offsets, lengths)."""
    idx = np.asarray(idx, np.int64)
    ln = np.asarray(lengths)[idx].astype(np.int32)
    off = np.zeros(idx.size, np.int64)
    if idx.size:
        off[1:] = np.cumsum(ln.astype(np.int64))[:-1]
    parts = [np.asarray(symbols)[o: o + t] for o, t in zip(np.asarray(offsets)[idx], ln)]
    sym = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
    return sym, off, ln


def allreduce_counts(tensors, group=None):
    """Sums the expected-count tensors over all ranks in place (the one
    collective of a data-parallel learning step)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors
