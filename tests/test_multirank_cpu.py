"""The multi-rank host logic on CPU.

A batch of independent graphs shards into contiguous graph ranges, one per
rank, with no exchange between ranks (`paper_2110_04865_gb300.shard`).  Two
gloo ranks (world size 2, 127.0.0.1) each solve their range -- with the
oracle, since this runs without a GPU -- and together they must give exactly
the per-graph totals, labels and masks of one process solving the whole
batch; the slowest-rank reduction the bench uses for its timings is checked
on the same ranks.

One graph shards by rows with one exchange per round: two gloo ranks run the
multilinear step and projection (Alg. 2) on their rows, join their projected
keys with a MIN all-reduce (order-preserving signed encoding of the keys),
and hook, break ties and shortcut on replicated parents; they must reach the
forest of one process."""
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


# ---- one graph, rows partitioned across ranks ------------------------------

def test_key_encoding_orders_like_unsigned():
    from paper_2110_04865_gb300.shard import key_to_signed, signed_to_key
    rng = np.random.default_rng(5)
    k = np.concatenate([rng.integers(0, 2**63, 500, dtype=np.uint64) << np.uint64(1),
                        np.array([0, 1, 2**63 - 1, 2**63, 2**64 - 1], dtype=np.uint64)])
    s = key_to_signed(k)
    assert s.dtype == np.int64 and np.array_equal(signed_to_key(s), k)
    order_u = np.argsort(k, kind="stable")
    assert np.array_equal(np.argsort(s, kind="stable"), order_u)
    assert int(s[k == 2**64 - 1][0]) == 2**63 - 1  # the identity stays the largest


def _hook_targets(r_key, ends, p_old):
    """Hook target of every root with a key: the parent, before hooking, of
    the endpoint of its edge that lies outside its star (the rule the hook
    kernel follows; the rank needs only the reduced key)."""
    INF = np.uint64(0xFFFFFFFFFFFFFFFF)
    r_par = np.full(len(p_old), -1, np.int64)
    for i in np.nonzero(r_key != INF)[0]:
        u, v = ends[int(r_key[i] & np.uint64(0xFFFFFFFF))]
        pu, pv = p_old[u], p_old[v]
        assert i in (pu, pv)
        r_par[i] = pv if pu == i else pu
    return r_par


def _row_worker(rank, ws, port, queue, n, src, dst, w):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import as_rounds
    from paper_2110_04865_gb300.shard import key_to_signed, row_ranges, signed_to_key
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        I, J, E = as_rounds.adjacency(n, src, dst)
        K = oracle.edge_keys(w, 0)[E]
        deg = np.bincount(I, minlength=n)
        row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
        r0, r1 = row_ranges(row_ptr, ws)[rank]
        mine = (I >= r0) & (I < r1)
        Il, Jl, Kl = I[mine], J[mine], K[mine]
        ends = np.stack([np.asarray(src, np.int64), np.asarray(dst, np.int64)], axis=1)
        p = np.arange(n, dtype=np.int64)
        mask = np.zeros(len(src), np.uint8)
        log = []
        for _ in range(64):
            p_old = p.copy()
            s = np.ones(n, bool)  # complete shortcutting: every tree is a star
            q_key, q_par = as_rounds.multilinear(n, Il, Jl, Kl, p, s)
            r_local, _ = as_rounds.project(n, q_key, q_par, p)
            t = torch.from_numpy(key_to_signed(r_local).copy())
            dist.all_reduce(t, op=dist.ReduceOp.MIN)  # the round's one exchange
            r_key = signed_to_key(t.numpy())
            r_par = _hook_targets(r_key, ends, p_old)
            p = as_rounds.hook(p, r_key, r_par)
            p, _, edges = as_rounds.tie_break(p, p_old, r_key)
            mask[edges] = 1
            p = as_rounds.csp_shortcut(p, p_old)
            log.append((int(len(edges)), r_local.copy(), r_key.copy()))
            if len(edges) == 0:
                break
        lab = np.full(n, np.iinfo(np.int64).max, np.int64)
        np.minimum.at(lab, p, np.arange(n))
        gathered = [None] * ws
        dist.all_gather_object(gathered, ((r0, r1), int(mine.sum()), mask, lab[p].astype(np.int32), log))
        if rank == 0:
            queue.put((gathered, row_ptr))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_solve_one_graph_by_row_partition():
    """Rows split across two ranks, one MIN all-reduce of the projected keys
    per round: both ranks reach the forest of one process (Kruskal's), and
    every round's reduced keys equal the projection over all rows."""
    mp = pytest.importorskip("torch.multiprocessing")
    n = 3000
    rng = np.random.default_rng(31)
    src = rng.integers(0, n, 9000).astype(np.int32)
    dst = rng.integers(0, n, 9000).astype(np.int32)
    w = ((rng.integers(0, 2**23, 9000) * 2 + 1) * 2.0**-24).astype(np.float32)  # ties occur
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_row_worker, args=(r, 2, port, queue, n, src, dst, w)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        gathered, row_ptr = queue.get(timeout=240)
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    assert all(pr.exitcode == 0 for pr in procs)
    (rg0, s0, mk0, lb0, log0), (rg1, s1, mk1, lb1, log1) = gathered
    assert rg0[0] == 0 and rg0[1] == rg1[0] and rg1[1] == n and s0 > 0 and s1 > 0
    assert s0 + s1 == int(row_ptr[-1])
    ref_mask, ref_lab, _ = oracle.kruskal(n, src, dst, w, 0)
    for mk, lb in ((mk0, lb0), (mk1, lb1)):
        assert np.array_equal(mk, ref_mask) and np.array_equal(lb, ref_lab)
    # the exchange: each round's reduced keys are the elementwise minimum of
    # the two ranks' partial projections, identical on both ranks
    assert len(log0) == len(log1)
    for (h0, pa, ra), (h1, pb, rb) in zip(log0, log1):
        assert h0 == h1 and np.array_equal(ra, rb)
        assert np.array_equal(ra, np.minimum(pa, pb))


def test_row_ranges_balance_slots_on_skewed_degrees():
    """Row ranges of an R-MAT-like degree sequence (a few hubs, many empty
    rows) cover the rows in order, and every rank's slots stay within one
    row's slots of the mean."""
    from paper_2110_04865_gb300.shard import row_ranges
    rng = np.random.default_rng(11)
    deg = (rng.pareto(1.2, 1 << 14) * 4).astype(np.int64)
    deg[rng.random(deg.size) < 0.3] = 0
    row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    for ws in (2, 3, 8):
        r = row_ranges(row_ptr, ws)
        assert r[0][0] == 0 and r[-1][1] == deg.size
        assert all(r[k][1] == r[k + 1][0] for k in range(ws - 1))
        slots = [int(row_ptr[b] - row_ptr[a]) for a, b in r]
        assert sum(slots) == int(row_ptr[-1])
        assert max(slots) <= row_ptr[-1] / ws + deg.max() + 1
