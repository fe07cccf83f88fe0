"""Sharding a batch of independent graphs across ranks (one process per GPU).

The graphs of a batch (msf_compute_batched) share no vertex, so a batch
splits into contiguous ranges of graphs with no exchange between ranks: each
rank solves its range with its own msf_compute_batched call and owns the
matching slices of the edge mask, the labels and the totals.  The ranges are
balanced by edge count (the round loop's work is proportional to the slots).
"""
from __future__ import annotations

import numpy as np


def shard_ranges(eoff, world_size: int) -> list[tuple[int, int]]:
    """Contiguous graph ranges [g0, g1), one per rank, covering 0..G-1 in
    order.  Rank r's range ends at the first graph boundary whose cumulative
    edge count reaches (r + 1) / world_size of the total, so every rank's
    edge count is within one graph of the mean."""
    eoff = np.asarray(eoff, dtype=np.int64)
    if world_size < 1:
        raise ValueError("world_size must be at least 1")
    G = len(eoff) - 1
    if G < 0:
        raise ValueError("eoff needs at least one entry")
    total = int(eoff[-1] - eoff[0])
    bounds = [0]
    for r in range(1, world_size):
        target = eoff[0] + (total * r) // world_size
        g = int(np.searchsorted(eoff, target, side="left"))
        bounds.append(min(max(g, bounds[-1]), G))
    bounds.append(G)
    return [(bounds[r], bounds[r + 1]) for r in range(world_size)]


def local_batch(voff, eoff, g0: int, g1: int):
    """The offsets of graphs [g0, g1) rebased to their own vertex and edge
    ranges, with those ranges: (voff_local, eoff_local, (v0, v1), (e0, e1)).
    Vertex ids in a batch are local to their graph, so the edge arrays'
    slice [e0, e1) is used as is."""
    voff = np.asarray(voff, dtype=np.int64)
    eoff = np.asarray(eoff, dtype=np.int64)
    v0, v1 = int(voff[g0]), int(voff[g1])
    e0, e1 = int(eoff[g0]), int(eoff[g1])
    return (np.ascontiguousarray(voff[g0:g1 + 1] - v0), np.ascontiguousarray(eoff[g0:g1 + 1] - e0),
            (v0, v1), (e0, e1))
