"""ORACLE (test infrastructure only): Prim's algorithm, one tree per component.

Used only to pin Kruskal: under a strict total edge order the minimum spanning
forest is unique (Sec. 1), so two unrelated greedy algorithms must agree edge
for edge.  Edges are compared by (ord(w), edge id) as in kruskal.c; a binary
heap holds the candidate edges leaving the growing tree.  Pure Python, for
small graphs.
"""
from __future__ import annotations

import heapq

import numpy as np

from . import edge_keys


def prim(n: int, src, dst, w, wtype: int) -> np.ndarray:
    """Returns the forest as a uint8 mask over the input edges."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keys = edge_keys(w, wtype)
    m = len(src)
    adj = [[] for _ in range(n)]
    for e in range(m):
        u, v = int(src[e]), int(dst[e])
        if u == v:
            continue
        adj[u].append((int(keys[e]), e, v))
        adj[v].append((int(keys[e]), e, u))
    mask = np.zeros(m, np.uint8)
    seen = [False] * n
    for start in range(n):
        if seen[start]:
            continue
        seen[start] = True
        heap = list(adj[start])
        heapq.heapify(heap)
        while heap:
            _, e, v = heapq.heappop(heap)
            if seen[v]:
                continue
            seen[v] = True
            mask[e] = 1
            for item in adj[v]:
                if not seen[item[2]]:
                    heapq.heappush(heap, item)
    return mask
