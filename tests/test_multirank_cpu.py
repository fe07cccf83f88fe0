"""The multi-rank host logic on CPU.

A batch of independent graphs shards into contiguous graph ranges, one per
rank, with no exchange between ranks (`paper_2110_04865_gb300.shard`).  Two
gloo ranks (world size 2, 127.0.0.1) each solve their range -- with the
oracle, since this runs without a GPU -- and together they must give exactly
the per-graph totals, labels and masks of one process solving the whole
batch; the slowest-rank reduction the bench uses for its timings is checked
on the same ranks."""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2110_04865_gb300.shard import local_batch, shard_ranges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_ranges_partition_and_balance():
    rng = np.random.default_rng(3)
    for G in (0, 1, 5, 64, 1000):
        sizes = rng.integers(0, 5000, G)
        eoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        biggest = int(sizes.max()) if G else 0
        for ws in (1, 2, 3, 8, 17):
            r = shard_ranges(eoff, ws)
            assert len(r) == ws
            assert r[0][0] == 0 and r[-1][1] == G
            assert all(a <= b for a, b in r)
            assert all(r[k][1] == r[k + 1][0] for k in range(ws - 1))
            edges = [int(eoff[b] - eoff[a]) for a, b in r]
            mean = int(eoff[-1]) / ws
            assert max(edges) <= mean + biggest + 1
    with pytest.raises(ValueError):
        shard_ranges([0, 3], 0)


def test_local_batch_rebases_offsets():
    voff = np.array([0, 4, 4, 10, 12], np.int64)
    eoff = np.array([0, 7, 7, 20, 21], np.int64)
    vo, eo, (v0, v1), (e0, e1) = local_batch(voff, eoff, 1, 3)
    assert (v0, v1, e0, e1) == (4, 10, 7, 20)
    assert vo.tolist() == [0, 0, 6] and eo.tolist() == [0, 0, 13]


def _solve_range(voff, eoff, s, d, w, g0, g1):
    """Per-graph oracle forests of graphs [g0, g1), from the rank's slices only."""
    vo, eo, (v0, v1), (e0, e1) = local_batch(voff, eoff, g0, g1)
    s, d, w = s[e0:e1], d[e0:e1], w[e0:e1]
    out = []
    for k in range(g1 - g0):
        a, b = int(eo[k]), int(eo[k + 1])
        mk, lb, tot = oracle.kruskal(int(vo[k + 1] - vo[k]), s[a:b], d[a:b], w[a:b], 0)
        out.append((mk, lb, tot))
    return out


def _worker(rank, ws, port, queue):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        import bench
        voff, eoff, s, d, w = synth.batch(24, nmax=2048, seed=9)[:5]
        g0, g1 = shard_ranges(eoff, ws)[rank]
        mine = _solve_range(voff, eoff, s, d, w, g0, g1)
        gathered = [None] * ws
        dist.all_gather_object(gathered, ((g0, g1), mine))
        slowest = bench.max_over_ranks(1.5 + rank, ws)
        if rank == 0:
            queue.put((gathered, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_solve_a_sharded_batch():
    mp = pytest.importorskip("torch.multiprocessing")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        gathered, slowest = queue.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert slowest == 2.5
    voff, eoff, s, d, w = synth.batch(24, nmax=2048, seed=9)[:5]
    whole = _solve_range(voff, eoff, s, d, w, 0, 24)
    (r0, part0), (r1, part1) = gathered
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == 24
    assert 0 < r0[1] < 24  # both ranks have work
    joined = part0 + part1
    assert len(joined) == len(whole)
    for (mk, lb, tot), (wmk, wlb, wtot) in zip(joined, whole):
        assert np.array_equal(mk, wmk) and np.array_equal(lb, wlb) and tot == wtot
