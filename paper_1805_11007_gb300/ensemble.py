"""Ensembles of independent replicates (the realisations the paper averages
over, Sect. 4): sharding across GPUs and host-side views of a batched
simulation.

Replicates are independent, so an ensemble shards across ranks with no data
exchange: each rank creates one batched simulation (``chemo_create_batch``)
of its own replicates. ``shard_replicates`` balances the particle count per
rank (largest replicate first onto the least-loaded rank; ties by rank), the
same on every rank, so no communication is needed to agree on it. The one
exchange is at the end: ``gather_replicates`` all-gathers each rank's
per-replicate rows (observables) into the global replicate order.
"""
from __future__ import annotations

import numpy as np


def shard_replicates(sizes, world: int) -> list:
    """Replicate indices of each of `world` ranks: greedy largest-first onto
    the rank with the fewest particles so far (deterministic). Every replicate
    lands on exactly one rank; each rank's list is in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64).reshape(-1)
    order = sorted(range(sizes.size), key=lambda r: (-int(sizes[r]), r))
    load = [0] * world
    out = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda q: (load[q], q))
        out[k].append(r)
        load[k] += int(sizes[r])
    return [sorted(v) for v in out]


def offsets(sizes) -> np.ndarray:
    """Start of each replicate in the concatenated arrays (R + 1 entries)."""
    sizes = np.asarray(sizes, dtype=np.int64).reshape(-1)
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def split(arr, sizes) -> list:
    """Per-replicate views of a concatenated array."""
    off = offsets(sizes)
    return [arr[off[r]:off[r + 1]] for r in range(len(off) - 1)]


def take(pos, sp, sizes, reps):
    """(sizes, pos, species) of the replicates `reps` (in that order)."""
    off = offsets(sizes)
    sizes = np.asarray(sizes, dtype=np.int64)
    idx = np.concatenate([np.arange(off[r], off[r + 1]) for r in reps]) if len(reps) else np.zeros(0, np.int64)
    return sizes[list(reps)], np.ascontiguousarray(pos[idx]), np.ascontiguousarray(sp[idx])


def gather_replicates(local_rows, sizes, world: int, rank: int, all_gather_object=None) -> np.ndarray:
    """Rows of every replicate in global replicate order, on every rank:
    `local_rows` holds one row per replicate of this rank's shard (in the
    shard's order, shard_replicates(sizes, world)[rank]); the shards' rows
    are exchanged with one all-gather (``all_gather_object`` of a process
    group, e.g. torch.distributed's; None with world == 1)."""
    shards = shard_replicates(sizes, world)
    local_rows = np.asarray(local_rows)
    if local_rows.shape[0] != len(shards[rank]):
        raise ValueError("one row per replicate of this rank's shard is required")
    if world == 1:
        parts = [local_rows]
    else:
        if all_gather_object is None:
            raise ValueError("a process group's all_gather_object is required for world > 1")
        parts = [None] * world
        all_gather_object(parts, local_rows)
    out = None
    for reps, rows in zip(shards, parts):
        rows = np.asarray(rows)
        if out is None:
            out = np.zeros((len(np.asarray(sizes).reshape(-1)),) + rows.shape[1:], rows.dtype)
        if len(reps):
            out[np.asarray(reps)] = rows
    return out
