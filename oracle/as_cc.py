"""ORACLE (test infrastructure only): Awerbuch-Shiloach connected components
in the linear-algebra form of Sec. 2.4, step by step.

Each round, with p_i the parent of i and s_i the star flag (Sec. 2.3):
  conditional hooking    p^h_i = min_j { p_j : a_ij present } for i in a star;
                         p_{p_i} <-min p^h_i  where p^h_i < p_i;
  starcheck;
  unconditional hooking  the same without the check, over the neighbours in
                         other trees (p_j != p_i), for vertices still in a
                         star (their trees hooked nowhere and nothing hooked
                         onto them);
  shortcutting           complete (every tree becomes a star), as in the
                         MSF method of Sec. 4.2.
The loop ends when a round changes no parent.  Readings: 0-based ids; "no
candidate" is +inf rather than 0; unconditional hooking skips neighbours in
the vertex's own tree (they would make a root its own parent).
"""
from __future__ import annotations

import numpy as np

from .as_rounds import adjacency, starcheck

BIG = np.iinfo(np.int64).max


def _hook(n, I, J, p, s, conditional: bool):
    """r_k = min p_j over edges (i, j) with i in a star, p_i = k and
    p_j < p_i (conditional) or p_j != p_i (unconditional); roots with a
    candidate take it as parent.  Returns (new p, number of hooks)."""
    pi, pj = p[I], p[J]
    ok = s[I] & ((pj < pi) if conditional else (pj != pi))
    r = np.full(n, BIG, np.int64)
    np.minimum.at(r, pi[ok], pj[ok])
    roots = np.nonzero(r != BIG)[0]
    p = p.copy()
    p[roots] = r[roots]
    return p, len(roots)


def complete_shortcut(p):
    while True:
        q = p[p]
        if np.array_equal(q, p):
            return p
        p = q


def as_cc(n: int, src, dst, max_rounds: int = 64):
    """Returns dict(labels (smallest vertex id per component), rounds, parent)."""
    I, J, _ = adjacency(n, src, dst)
    p = np.arange(n, dtype=np.int64)
    rounds = 0
    while True:
        if rounds == max_rounds:
            raise RuntimeError("round limit")
        rounds += 1
        p_old = p.copy()
        p, h1 = _hook(n, I, J, p, starcheck(p), conditional=True)
        p, h2 = _hook(n, I, J, p, starcheck(p), conditional=False)
        p = complete_shortcut(p)
        if np.array_equal(p, p_old):
            break
    lab = np.full(n, BIG, np.int64)
    np.minimum.at(lab, p, np.arange(n))
    return dict(labels=lab[p].astype(np.int32), rounds=rounds, parent=p)
