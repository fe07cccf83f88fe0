"""ORACLE (test infrastructure only): Awerbuch-Shiloach connected components
in the linear-algebra form of Sec. 2.4, step by step.

Each round, with p_i the parent of i and s_i the star flag (Sec. 2.3):
  conditional hooking    p^h_i = min_j { p_j : a_ij present } for i in a star;
                         p_{p_i} <-min p^h_i  where p^h_i < p_i;
  starcheck;
  unconditional hooking  the same without the check p^h_i < p_i, for
                         vertices i still in a star, over the neighbours j
                         whose tree is not a star;
  shortcutting           complete (every tree becomes a star), as in the
                         MSF method of Sec. 4.2.
The loop ends when a round changes no parent.

Readings (the paper states the unconditional step only as "the same
without the check"): 0-based ids; "no candidate" is +inf rather than 0; the
unconditional step hooks a star only onto a neighbour in a tree that is not
a star, the form of the connectivity algorithm the section restates (Azad
and Buluc's LACC).  Without that restriction two stars left adjacent after
conditional hooking (one of them grown by a single vertex that hooked onto
it and left it a star) hook onto each other and form a 2-cycle; a
non-star tree never moves during the unconditional step, so with it no
cycle can form.  Termination is unaffected: in a round without any hook
every tree is a star and no star has a neighbour with a smaller root, so no
edge leaves any tree.
"""
from __future__ import annotations

import numpy as np

from .as_rounds import adjacency, starcheck

BIG = np.iinfo(np.int64).max


def _hook(n, I, J, p, s, conditional: bool):
    """r_k = min p_j over edges (i, j) with i in a star, p_i = k, and
    p_j < p_i (conditional) or j's tree not a star (unconditional); roots
    with a candidate take it as parent.  Returns (new p, number of hooks)."""
    pi, pj = p[I], p[J]
    ok = s[I] & ((pj < pi) if conditional else ~s[J])
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


def labels_of(p):
    """Smallest vertex id of each vertex's tree (p: every tree a star)."""
    n = len(p)
    lab = np.full(n, BIG, np.int64)
    np.minimum.at(lab, p, np.arange(n))
    return lab[p].astype(np.int32)


def as_cc(n: int, src, dst, max_rounds: int = 64, stop_after: int | None = None):
    """Returns dict(labels (smallest vertex id per tree), rounds, parent,
    history): history[k] holds, for round k + 1, the parents after
    conditional hooking, the star flags after it, the parents after
    unconditional hooking and after shortcutting.  stop_after=k stops after
    round k (the partial forest's labels)."""
    I, J, _ = adjacency(n, src, dst)
    p = np.arange(n, dtype=np.int64)
    rounds = 0
    history = []
    while True:
        if rounds == max_rounds:
            raise RuntimeError("round limit")
        if stop_after is not None and rounds == stop_after:
            break
        rounds += 1
        p_old = p.copy()
        p_c, _ = _hook(n, I, J, p, starcheck(p), conditional=True)
        s_c = starcheck(p_c)
        p_u, _ = _hook(n, I, J, p_c, s_c, conditional=False)
        p = complete_shortcut(p_u)
        history.append(dict(cond=p_c, star=s_c, uncond=p_u, shortcut=p))
        if np.array_equal(p, p_old):
            break
    return dict(labels=labels_of(p), rounds=rounds, parent=p, history=history)
