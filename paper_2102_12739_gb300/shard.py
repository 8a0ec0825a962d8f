"""Sharding of a degridding job across GPUs (one process per GPU).

Subgrids are independent and every visibility belongs to exactly one subgrid
(Section "Implementation": S subgrids, each with its own list of
visibilities), so a job splits across ranks by whole subgrids with no
exchange on the data path: each rank degrids (or grids) the subgrids it owns
and writes its own visibilities.  The only cross-rank operations are
host-side: agreeing on the partition, and reducing timings and counts.

Partition: greedy longest-processing-time on the visibility counts (largest
subgrid first, each to the currently lightest rank; ties to the lower rank),
which keeps the per-rank visibility totals within one subgrid of each other.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence

import numpy as np


def partition_subgrids(counts: Sequence[int], world: int) -> List[np.ndarray]:
    """Subgrid indices owned by each of `world` ranks (sorted ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    counts = np.asarray(counts, dtype=np.int64)
    order = np.argsort(-counts, kind="stable")
    heap = [(0, r) for r in range(world)]
    owned: List[list] = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        owned[r].append(int(s))
        heapq.heappush(heap, (load + int(counts[s]), r))
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def shard_offsets(vis_offsets: Sequence[int], owned: Sequence[int]):
    """Visibility index ranges and local offsets of the owned subgrids.

    Returns (global_ranges [k][2], local_offsets [k + 1]): the rank's inputs
    are the concatenation of uvw[lo:hi] over its ranges, delimited by the
    local offsets.
    """
    offs = np.asarray(vis_offsets, dtype=np.int64)
    owned = np.asarray(owned, dtype=np.int64)
    ranges = np.stack([offs[owned], offs[owned + 1]], axis=1) if len(owned) else np.zeros((0, 2), np.int64)
    local = np.zeros(len(owned) + 1, dtype=np.int64)
    np.cumsum(ranges[:, 1] - ranges[:, 0], out=local[1:])
    return ranges, local


def gather_uvw(uvw: np.ndarray, ranges: np.ndarray) -> np.ndarray:
    if len(ranges) == 0:
        return np.zeros((0, 3), dtype=np.float64)
    return np.ascontiguousarray(np.concatenate([uvw[lo:hi] for lo, hi in ranges]))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. a step time) over the process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: int, device=None) -> int:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(value)
    t = torch.tensor([int(value)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())
