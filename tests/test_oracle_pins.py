"""Pins for the CPU oracle against things other than itself (no GPU).

The forest Kruskal returns is checked against Prim, against exhaustive search,
against scipy's minimum_spanning_tree, against the cut and cycle properties
(Sec. 1), against closed forms, against hand-worked examples in tests/golden/,
and against Algorithm 2 run step by step.  The exact total is checked against
rational arithmetic.  Each check is chosen so that a plausible mistake (a
dropped tie-break, a wrong comparison, a lost edge) fails at least one; the
planted-mistake tests at the end show that they do.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree

import oracle
from oracle import as_rounds, edge_keys
from oracle.brute import brute_force
from oracle.prim import prim
from golden_io import all_fixtures


def rand_graph(rng, n, m, wtype, levels=None, negative=False):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if wtype == 0:
        if levels:
            vals = rng.choice(np.linspace(-1 if negative else 0.0625, 1, levels), m)
            w = vals.astype(np.float32)
        else:
            w = rng.random(m).astype(np.float32)
            if negative:
                w -= np.float32(0.5)
    else:
        w = rng.integers(1, (levels or 1000) + 1, m).astype(np.uint32)
    return src, dst, w


def components(n, src, dst):
    a = sp.coo_matrix((np.ones(len(src)), (src, dst)), shape=(n, n))
    return connected_components(a, directed=False)


CASES = [(n, m, wt, lv) for n, m in [(1, 0), (2, 1), (5, 3), (12, 30), (40, 60), (64, 400), (300, 900)]
         for wt in (0, 1) for lv in (None, 3)]


@pytest.mark.parametrize("n,m,wtype,levels", CASES)
def test_kruskal_equals_prim(n, m, wtype, levels):
    rng = np.random.default_rng(n * 1000 + m + wtype + (levels or 0))
    src, dst, w = rand_graph(rng, n, m, wtype, levels)
    mask, labels, total = oracle.kruskal(n, src, dst, w, wtype)
    assert np.array_equal(mask, prim(n, src, dst, w, wtype))


@pytest.mark.parametrize("seed", range(40))
def test_kruskal_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 15))
    wtype = seed % 2
    src, dst, w = rand_graph(rng, n, m, wtype, levels=3, negative=(wtype == 0))
    mask, labels, total = oracle.kruskal(n, src, dst, w, wtype)
    bmask, bweight = brute_force(n, src, dst, w, wtype)
    assert np.array_equal(mask, bmask)
    # least total weight over all spanning forests (rank order == weight order)
    assert total == pytest.approx(bweight, abs=1e-9)


@pytest.mark.parametrize("n,density", [(50, 0.2), (400, 0.02), (2000, 0.003)])
def test_kruskal_equals_scipy_distinct_weights(n, density):
    rng = np.random.default_rng(n)
    # simple graph (no loops, no parallel edges), distinct positive weights
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < density
    src, dst = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    perm = rng.permutation(len(src))
    w = ((perm + 1) * 2.0 ** -20).astype(np.float32)
    mask, labels, total = oracle.kruskal(n, src, dst, w, 0)
    t = minimum_spanning_tree(sp.coo_matrix((w.astype(np.float64), (src, dst)), shape=(n, n))).tocoo()
    chosen = set(zip(np.minimum(t.row, t.col).tolist(), np.maximum(t.row, t.col).tolist()))
    ours = set(zip(src[mask == 1].tolist(), dst[mask == 1].tolist()))
    assert chosen == ours
    assert total == math.fsum(t.data.tolist())


@pytest.mark.parametrize("n,m", [(1, 0), (10, 0), (100, 50), (1000, 800), (1000, 5000), (5000, 4000)])
def test_forest_size_and_canonical_labels(n, m):
    rng = np.random.default_rng(m)
    src, dst, w = rand_graph(rng, n, m, 0, levels=5)
    mask, labels, total = oracle.kruskal(n, src, dst, w, 0)
    ncomp, comp = components(n, src, dst)
    assert int(mask.sum()) == n - ncomp
    assert mask[src == dst].sum() == 0
    # labels: equal iff same component, and the smallest vertex of it
    for c in range(ncomp):
        members = np.nonzero(comp == c)[0]
        assert np.all(labels[members] == members.min())
    # forest edges alone span the same components
    fc, fcomp = components(n, src[mask == 1], dst[mask == 1])
    assert fc == ncomp


def _tree_path_max(n, fsrc, fdst, fkey, u, v):
    adj = [[] for _ in range(n)]
    for a, b, k in zip(fsrc, fdst, fkey):
        adj[a].append((b, k))
        adj[b].append((a, k))
    best = {u: 0}
    stack = [u]
    while stack:
        x = stack.pop()
        for y, k in adj[x]:
            if y not in best:
                best[y] = max(best[x], k)
                stack.append(y)
    return best.get(v)


@pytest.mark.parametrize("seed", range(6))
def test_cut_and_cycle_properties(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = 60, 150
    src, dst, w = rand_graph(rng, n, m, seed % 2, levels=4)
    mask, labels, total = oracle.kruskal(n, src, dst, w, seed % 2)
    keys = edge_keys(w, seed % 2).astype(object)
    F = np.nonzero(mask)[0]
    # cut property: removing forest edge e splits its tree into S and T;
    # e is the least-key edge with one end in S and the other in T
    for e in F:
        rest = [f for f in F if f != e]
        _, comp = components(n, src[rest], dst[rest])
        cs, ct = comp[src[e]], comp[dst[e]]
        crossing = [f for f in range(m) if {comp[src[f]], comp[dst[f]]} == {cs, ct}]
        assert min(crossing, key=lambda f: keys[f]) == e
    # cycle property: a non-forest, non-loop edge is the largest key on the
    # cycle it closes
    for e in range(m):
        if mask[e] or src[e] == dst[e]:
            continue
        mx = _tree_path_max(n, src[F], dst[F], keys[F], int(src[e]), int(dst[e]))
        assert mx is not None and mx < keys[e]


def test_closed_forms():
    # a tree input keeps every edge
    rng = np.random.default_rng(7)
    n = 200
    parent = np.array([rng.integers(0, v) for v in range(1, n)])
    src = np.arange(1, n, dtype=np.int32)
    dst = parent.astype(np.int32)
    w = rng.random(n - 1).astype(np.float32)
    mask, labels, total = oracle.kruskal(n, src, dst, w, 0)
    assert mask.all() and np.all(labels == 0)
    # complete graph, all weights equal: the n-1 lowest indices that close no
    # cycle, i.e. the star of vertex 0 when edges are listed (i<j) row by row
    n = 30
    iu, ju = np.triu_indices(n, 1)
    w = np.full(len(iu), 7, np.uint32)
    mask, labels, total = oracle.kruskal(n, iu.astype(np.int32), ju.astype(np.int32), w, 1)
    assert np.array_equal(mask.astype(bool), iu == 0)
    assert total == 7 * (n - 1)
    # path with increasing weights and no other edges: every edge
    n = 100
    mask, labels, total = oracle.kruskal(n, np.arange(n - 1, dtype=np.int32),
                                         np.arange(1, n, dtype=np.int32),
                                         np.arange(1, n, dtype=np.uint32), 1)
    assert mask.all() and total == n * (n - 1) // 2
    # cycle with increasing weights drops exactly the heaviest edge
    mask, labels, total = oracle.kruskal(n, np.arange(n, dtype=np.int32),
                                         ((np.arange(n) + 1) % n).astype(np.int32),
                                         np.arange(1, n + 1, dtype=np.uint32), 1)
    assert mask[:-1].all() and mask[-1] == 0
    # isolated vertices keep their own label
    mask, labels, total = oracle.kruskal(5, np.array([1], np.int32), np.array([3], np.int32),
                                         np.array([0.5], np.float32), 0)
    assert list(labels) == [0, 1, 2, 1, 4] and total == 0.5
    # uniform-weight 3-D grid: a spanning tree of weight w (n - 1)
    import synth
    s, d, _ = synth.grid3d(6, 5, 4, wtype=1)
    w = np.full(len(s), 3, np.uint32)
    mask, labels, total = oracle.kruskal(120, s, d, w, 1)
    assert mask.sum() == 119 and total == 3 * 119 and np.all(labels == 0)


@pytest.mark.parametrize("fx", all_fixtures(), ids=lambda f: f["name"])
def test_golden_hand_worked(fx):
    mask, labels, total = oracle.kruskal(fx["n"], fx["src"], fx["dst"], fx["w"], fx["wtype"])
    assert np.array_equal(mask, fx["mask"])
    assert np.array_equal(labels, fx["labels"])
    assert total == fx["total"]
    r = as_rounds.as_msf(fx["n"], fx["src"], fx["dst"], fx["w"], fx["wtype"])
    assert np.array_equal(r["mask"], fx["mask"])
    if "rounds" in fx:
        assert r["rounds"] == fx["rounds"]
    for k, p in fx["parent"].items():
        assert np.array_equal(r["history"][k - 1], p)


def test_exact_total_against_rationals():
    rng = np.random.default_rng(3)
    for trial in range(30):
        k = int(rng.integers(0, 400))
        mant = rng.integers(1, 1 << 24, k)
        expo = rng.integers(-60, 60, k)
        sign = rng.choice([-1.0, 1.0], k)
        v = (sign * mant * np.exp2(expo.astype(np.float64))).astype(np.float32)
        exact = sum((Fraction(float(x)) for x in v), Fraction(0))
        assert oracle.exact_total(v, 0) == float(exact)   # Fraction -> float rounds to nearest
    # sums that cancel catastrophically
    v = np.array([2.0 ** 100, 1.0, -(2.0 ** 100), 2.0 ** -100], np.float32)
    assert oracle.exact_total(v, 0) == 1.0 + 2.0 ** -100
    # integer weights
    u = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64).astype(np.uint32)
    assert oracle.exact_total(u, 1) == float(sum(int(x) for x in u))
    assert math.isnan(oracle.exact_total(np.array([np.inf, -np.inf], np.float32), 0))


@pytest.mark.parametrize("seed", range(12))
def test_algorithm2_reaches_kruskal(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(2, 400))
    m = int(rng.integers(0, 4 * n))
    wtype = seed % 2
    src, dst, w = rand_graph(rng, n, m, wtype, levels=(None if seed % 3 else 4))
    mask, labels, total = oracle.kruskal(n, src, dst, w, wtype)
    r = as_rounds.as_msf(n, src, dst, w, wtype)
    assert np.array_equal(r["mask"], mask)
    assert np.array_equal(r["labels"], labels)
    assert r["total"] == total
    # complete shortcutting: every tree with an outgoing edge hooks or is
    # hooked onto, so at least half of them hook (Sec. 4.2) and the number
    # of rounds is logarithmic
    for h, t in zip(r["hooks"], r["trees"]):
        assert 2 * h >= t
    assert r["rounds"] <= math.ceil(math.log2(max(n, 2))) + 2


def test_starcheck_small_forests():
    # a star rooted at 0, and a path 3 -> 2 -> 1 -> 1 (not a star)
    p = np.array([0, 1, 1, 2, 0])
    s = as_rounds.starcheck(p)
    assert list(s) == [True, False, False, False, True]
    assert as_rounds.starcheck(np.arange(6)).all()


def test_multilinear_one_round_definition():
    # Sec. 3.1: q_i = least (a_ij, p_j) over j with p_i != p_j, i in a star
    rng = np.random.default_rng(11)
    n, m = 50, 200
    src, dst, w = rand_graph(rng, n, m, 0, levels=6)
    I, J, E = as_rounds.adjacency(n, src, dst)
    K = edge_keys(w, 0)[E]
    p = rng.integers(0, 5, n)
    p[:5] = np.arange(5)
    s = np.ones(n, bool)
    q_key, q_par = as_rounds.multilinear(n, I, J, K, p, s)
    for i in range(n):
        cands = [(int(K[t]), int(p[J[t]])) for t in range(len(I)) if I[t] == i and p[i] != p[J[t]]]
        if cands:
            assert (int(q_key[i]), int(q_par[i])) == min(cands)
        else:
            assert q_key[i] == as_rounds.INF and q_par[i] == -1


# ---- planted mistakes: the pins above must catch each of them ---------------

def test_planted_dropped_tie_break_is_caught(monkeypatch):
    """Tie ids dropped from the key (all equal weights look alike): Algorithm 2
    then forms longer cycles or picks different edges, and disagrees with
    Kruskal on a tied graph."""
    def bad_keys(w, wtype):
        o = oracle.ord_words(oracle.weight_words(w, wtype), wtype).astype(np.uint64)
        return o << np.uint64(32)
    monkeypatch.setattr(as_rounds, "edge_keys", bad_keys)
    src = np.array([0, 1, 0, 2], np.int32)
    dst = np.array([1, 2, 2, 3], np.int32)
    w = np.ones(4, np.uint32)
    mask, labels, total = oracle.kruskal(4, src, dst, w, 1)
    try:
        r = as_rounds.as_msf(4, src, dst, w, 1)
        caught = not np.array_equal(r["mask"], mask)
    except (RuntimeError, IndexError):
        caught = True
    assert caught


def test_planted_reversed_tie_break_is_caught(monkeypatch):
    """Tie breaking that keeps the larger root (i > p_i) still forms a forest
    but the golden round-by-round parents disagree."""
    def bad_tie_break(p, p_old, r_key):
        n = len(p)
        i = np.arange(n)
        root = p_old == i
        t = root & (i > p) & (p[p] == i)
        p = np.where(t, i, p)
        add = root & (r_key != as_rounds.INF) & ~t
        return p, t, (r_key[add] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    monkeypatch.setattr(as_rounds, "tie_break", bad_tie_break)
    fx = [f for f in all_fixtures() if f["name"] == "tie_break_two_rounds.txt"][0]
    r = as_rounds.as_msf(fx["n"], fx["src"], fx["dst"], fx["w"], fx["wtype"])
    assert not np.array_equal(r["history"][0], fx["parent"][1])


def test_planted_inexact_sum_is_caught():
    """Plain float32 accumulation fails the rational-arithmetic pin."""
    v = np.array([2.0 ** 30, 1.0, -(2.0 ** 30), 0.5], np.float32)
    naive = float(np.float32(np.float32(np.float32(v[0] + v[1]) + v[2]) + v[3]))
    exact = float(sum((Fraction(float(x)) for x in v), Fraction(0)))
    assert naive != exact and oracle.exact_total(v, 0) == exact


@pytest.mark.parametrize("seed", range(8))
def test_original_schedule_reaches_kruskal(seed):
    """Algorithm 1's schedule (starcheck, one shortcut step per round) reaches
    the same forest; it needs at least as many rounds as complete shortcutting
    and stays within the log_{3/2} n bound of Sec. 2.3 (plus the final check)."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 1500))
    m = int(rng.integers(0, 4 * n))
    wtype = seed % 2
    src, dst, w = rand_graph(rng, n, m, wtype, levels=(3 if seed % 2 else None))
    mask, labels, total = oracle.kruskal(n, src, dst, w, wtype)
    a = as_rounds.as_msf(n, src, dst, w, wtype, mode="original", max_rounds=500)
    c = as_rounds.as_msf(n, src, dst, w, wtype)
    assert np.array_equal(a["mask"], mask) and np.array_equal(a["labels"], labels) and a["total"] == total
    assert a["rounds"] >= c["rounds"]
    assert a["rounds"] <= math.ceil(math.log(max(n, 2), 1.5)) + 2


def test_partial_rounds_nest():
    rng = np.random.default_rng(5)
    src, dst, w = rand_graph(rng, 300, 900, 0)
    full = as_rounds.as_msf(300, src, dst, w, 0)
    prev = np.zeros(900, np.uint8)
    for k in range(1, full["rounds"] + 1):
        part = as_rounds.as_msf(300, src, dst, w, 0, stop_after=k)
        assert part["rounds"] == k
        assert np.all(part["mask"] >= prev)   # forest edges only accumulate
        assert np.array_equal(part["history"][-1], full["history"][k - 1])
        prev = part["mask"]
    assert np.array_equal(prev, full["mask"])


@pytest.mark.parametrize("seed", range(8))
def test_connectivity_oracle_matches_scipy(seed):
    """Sec. 2.4 step by step gives the connected components (scipy's BFS-based
    labels, made canonical), with a logarithmic number of rounds."""
    from oracle import as_cc
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 3 * n))
    src, dst, _ = rand_graph(rng, n, m, 0)
    r = as_cc.as_cc(n, src, dst)
    ncomp, comp = components(n, src, dst)
    canon = np.zeros(n, np.int64)
    for c in range(ncomp):
        members = np.nonzero(comp == c)[0]
        canon[members] = members.min()
    assert np.array_equal(r["labels"], canon)
    assert r["rounds"] <= math.ceil(math.log2(max(n, 2))) + 2


# ---- connectivity (Sec. 2.4) -------------------------------------------------------

def _cc_fixture():
    from golden_io import connectivity_fixtures
    return connectivity_fixtures()[0]


def test_connectivity_oracle_hand_worked_rounds():
    """The step oracle follows the hand-worked rounds of the fixture exactly:
    parents after conditional hooking, star flags, parents after unconditional
    hooking and after shortcutting, round by round."""
    from oracle import as_cc
    fx = _cc_fixture()
    r = as_cc.as_cc(fx["n"], fx["src"], fx["dst"])
    assert r["rounds"] == fx["rounds"]
    assert np.array_equal(r["labels"], fx["labels"])
    for k, par in fx["parent"].items():
        h = r["history"][k - 1]
        assert np.array_equal(h["shortcut"], par), k
        if k in fx["cond"]:
            assert np.array_equal(h["cond"], fx["cond"][k]), k
            assert np.array_equal(h["star"].astype(np.int64), fx["star"][k]), k
            assert np.array_equal(h["uncond"], fx["uncond"][k]), k
        part = as_cc.as_cc(fx["n"], fx["src"], fx["dst"], stop_after=k)
        assert np.array_equal(part["parent"], par), k


def _acyclic(p):
    """True iff following parents from every vertex ends at a root (a vertex
    that is its own parent): after enough doubling steps every vertex must
    point at one."""
    q = p.copy()
    for _ in range(int(np.ceil(np.log2(max(len(p), 2)))) + 1):
        q = q[q]
    return bool(np.all(p[q] == q))


@pytest.mark.parametrize("seed", range(12))
def test_connectivity_hooks_keep_a_forest(seed):
    """Sec. 2.4's hooking rules, checked on the oracle's own trajectory:
    conditional hooks point at a smaller root; unconditional hooks start at a
    root whose tree is a star after the conditional step and end in a tree
    that is not a star; after either step the parent graph has no cycle."""
    from oracle import as_cc
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(2, 3000))
    m = int(rng.integers(0, 3 * n))
    src, dst, _ = rand_graph(rng, n, m, 0)
    r = as_cc.as_cc(n, src, dst)
    p = np.arange(n)
    for h in r["history"]:
        moved = np.nonzero(h["cond"] != p)[0]
        assert np.all(p[moved] == moved) and np.all(h["cond"][moved] < moved)
        assert _acyclic(h["cond"])
        um = np.nonzero(h["uncond"] != h["cond"])[0]
        assert np.all(h["cond"][um] == um) and np.all(h["star"][um])
        assert not np.any(h["star"][h["uncond"][um]])
        assert _acyclic(h["uncond"])
        p = h["shortcut"]
        assert np.all(p[p] == p)


def test_planted_unrestricted_unconditional_hooking_is_caught(monkeypatch):
    """Unconditional hooking onto any neighbour in another tree (star or not)
    makes the stars {1} and {0,2} of the fixture hook onto each other: the
    hand-worked parents and the no-cycle invariant both catch it."""
    from oracle import as_cc

    def loose_hook(n, I, J, p, s, conditional):
        pi, pj = p[I], p[J]
        ok = s[I] & ((pj < pi) if conditional else (pj != pi))
        r = np.full(n, as_cc.BIG, np.int64)
        np.minimum.at(r, pi[ok], pj[ok])
        roots = np.nonzero(r != as_cc.BIG)[0]
        p = p.copy()
        p[roots] = r[roots]
        return p, len(roots)

    fx = _cc_fixture()
    monkeypatch.setattr(as_cc, "_hook", loose_hook)
    I, J, _ = as_rounds.adjacency(fx["n"], fx["src"], fx["dst"])
    p = np.arange(fx["n"])
    pc, _ = as_cc._hook(fx["n"], I, J, p, as_rounds.starcheck(p), True)
    pu, _ = as_cc._hook(fx["n"], I, J, pc, as_rounds.starcheck(pc), False)
    assert not np.array_equal(pu, fx["uncond"][1])
    assert not _acyclic(pu)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_all_cores_variant_equals_kruskal(threads):
    """The all-cores CPU baseline (keys built and radix-sorted on several
    threads, then the same sequential scan) returns exactly the forest, labels
    and total of the single-threaded oracle, ties and self-loops included."""
    rng = np.random.default_rng(40 + threads)
    for n, m, wtype, levels in [(1, 0, 0, None), (50, 400, 1, 3), (3000, 20000, 0, 5), (2000, 9000, 0, None)]:
        src, dst, w = rand_graph(rng, n, m, wtype, levels)
        a = oracle.kruskal(n, src, dst, w, wtype)
        b = oracle.kruskal_mt(n, src, dst, w, wtype, threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
