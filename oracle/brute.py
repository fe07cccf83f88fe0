"""ORACLE (test infrastructure only): exhaustive search over spanning forests.

For graphs with at most 8 vertices and about 14 non-loop edges, every edge
subset of size n - c (c = number of connected components) that contains no
cycle is a spanning forest.  Weights are replaced by their rank in the strict
(ord(w), edge id) order, which makes them distinct without changing which
forest a greedy algorithm picks; the forest with the least rank sum is then
unique and must equal the one Kruskal returns.  Its true weight must also be
the least true weight over all spanning forests.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import edge_keys


def _components(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    comp = [-1] * n
    c = 0
    for s in range(n):
        if comp[s] >= 0:
            continue
        stack = [s]
        comp[s] = c
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if comp[y] < 0:
                    comp[y] = c
                    stack.append(y)
        c += 1
    return c, comp


def _acyclic(n, edges):
    up = list(range(n))

    def find(x):
        while up[x] != x:
            x = up[x]
        return x

    for u, v in edges:
        a, b = find(u), find(v)
        if a == b:
            return False
        up[a] = b
    return True


def brute_force(n: int, src, dst, w, wtype: int):
    """Returns (mask of the least-rank forest, least true weight over all forests)."""
    m = len(src)
    keys = edge_keys(w, wtype)
    cand = [e for e in range(m) if int(src[e]) != int(dst[e])]
    if len(cand) > 16:
        raise ValueError("too many edges for exhaustive search")
    rank = {e: r for r, e in enumerate(sorted(cand, key=lambda e: int(keys[e])))}
    c, _ = _components(n, [(int(src[e]), int(dst[e])) for e in cand])
    k = n - c
    best_rank, best_set, best_weight = None, None, None
    wv = np.asarray(w)
    for sub in itertools.combinations(cand, k):
        edges = [(int(src[e]), int(dst[e])) for e in sub]
        if not _acyclic(n, edges):
            continue
        rs = sum(rank[e] for e in sub)
        if best_rank is None or rs < best_rank:
            best_rank, best_set = rs, sub
        tw = sum(float(wv[e]) for e in sub)
        if best_weight is None or tw < best_weight:
            best_weight = tw
    mask = np.zeros(m, np.uint8)
    for e in best_set or ():
        mask[e] = 1
    return mask, (best_weight if best_weight is not None else 0.0)
