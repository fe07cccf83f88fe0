"""Sharding across ranks (one process per GPU).

Batches: the graphs of a batch (msf_compute_batched) share no vertex, so a
batch splits into contiguous ranges of graphs with no exchange between ranks:
each rank solves its range with its own msf_compute_batched call and owns the
matching slices of the edge mask, the labels and the totals.  The ranges are
balanced by edge count (the round loop's work is proportional to the slots).

One graph: a 1-D partition of the CSR by slot count (the single-process
counterpart of Sec. 4.1's distribution of A), parents replicated.  Every
round each rank runs the multilinear step and projection (Alg. 2) on its part
only (msf_min_edge_part), a MIN all-reduce of the n projected keys joins the
ranks, and every rank then hooks, breaks ties and shortcuts redundantly on
the replicated parents (msf_apply_round): every rank derives the same changed
parents from the same reduced keys, so Algorithm 3's all-gather of the
changed map needs no message and its chase runs locally.  The keys are
unsigned 64-bit words; `key_to_signed` maps them, order preserving, onto the
signed 64-bit integers that collective MIN reductions take.
`solve_partitioned` drives that loop through the library with a
caller-supplied MIN all-reduce; the rest of this module is host logic.
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


def row_ranges(row_ptr, world_size: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [r0, r1), one per rank, of a CSR with offsets
    row_ptr (n + 1 entries), balanced by slot count: each rank's slots are
    within one row's slots of the mean."""
    return shard_ranges(row_ptr, world_size)


_SIGN = np.uint64(1) << np.uint64(63)


def key_to_signed(keys) -> np.ndarray:
    """Unsigned 64-bit keys -> signed 64-bit integers in the same order
    (the top bit flipped), so that a signed MIN reduction yields the
    unsigned minimum; the identity key 2^64 - 1 maps to 2^63 - 1."""
    k = np.asarray(keys, dtype=np.uint64)
    return (k ^ _SIGN).view(np.int64)


def signed_to_key(x) -> np.ndarray:
    """Inverse of key_to_signed."""
    return np.asarray(x, dtype=np.int64).view(np.uint64) ^ _SIGN


def solve_partitioned(handle: int, n: int, m: int, part: int, nparts: int, allreduce_min, device,
                      stream: int = 0, max_rounds: int = 64):
    """Forest of one built graph (msf_build_csr handle) by the partitioned
    round loop: this process sweeps part `part` of `nparts` slot ranges, and
    `allreduce_min(x)` must return the elementwise minimum of the int64 numpy
    array x over all parts (for instance a torch.distributed MIN all-reduce
    of a CPU tensor).  Returns (edge_mask, labels) as device tensors and the
    number of rounds; every process ends with the same result."""
    import torch

    from . import _abi
    parent = torch.arange(n, dtype=torch.int32, device=device)
    r = torch.empty(n, dtype=torch.int64, device=device)
    mask = torch.zeros(m, dtype=torch.uint8, device=device)
    labels = torch.empty(n, dtype=torch.int32, device=device)
    rounds = 0
    while True:
        if rounds == max_rounds:
            raise RuntimeError("round limit reached")
        rounds += 1
        _abi.msf_min_edge_part(handle, parent.data_ptr(), part, nparts, r.data_ptr(), stream)
        red = allreduce_min(key_to_signed(r.cpu().numpy().view(np.uint64)))
        r.copy_(torch.from_numpy(signed_to_key(red).view(np.int64)))
        hooks = _abi.msf_apply_round(handle, r.data_ptr(), parent.data_ptr(), mask.data_ptr(), labels.data_ptr(),
                                     stream)
        if hooks == 0:
            return mask, labels, rounds
