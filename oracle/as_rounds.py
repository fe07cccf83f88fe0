"""ORACLE (test infrastructure only): Algorithm 2 (Awerbuch-Shiloach with
linear algebra, Sec. 3.2) with complete shortcutting (Sec. 4.2, Algorithm 3),
one step at a time in the paper's order and notation.

Readings taken where the paper is silent or garbled:
  * EDGE elements carry (weight, parent); the weight is made strict by the
    tie id, i.e. the element is (key(e), p_j) with key(e) = ord(w_e)*2^32 + e.
    MinWeight picks the least key.  The identity (inf, 0) is (INF, -1).
  * Vertices are 0-based; "no parent" is -1 instead of 0.
  * The weight update adds r_i only for star roots that hooked (r_i not the
    identity) and were not reset by tie breaking.  The forest edge is
    recorded too.
  * The shortcut step leaves star vertices' parents unchanged (as in
    Algorithm 1; the printed rule sets them to 0), and the shortcut is complete: Algorithm 3 chases every vertex's parent
    through the map of roots whose parent changed this round.
  * The loop stops once a round leaves p unchanged (the loop test).

``as_msf(mode="original")`` runs the original schedule instead: a real
starcheck before hooking and before shortcutting, and one shortcut step per
round (Algorithm 1).

Each step is a separate function so the GPU kernels can be checked one at a
time: ``multilinear`` (multilinear step), ``project`` (projection onto the
root), ``hook`` (hooking), ``tie_break`` (tie breaking and the weight
update), ``csp_shortcut`` (Algorithm 3) and
``starcheck`` (Sec. 2.3).
"""
from __future__ import annotations

import numpy as np

from . import edge_keys, exact_total, weight_words

INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def adjacency(n: int, src, dst):
    """Both directions of every non-loop edge: rows I, columns J, edge ids E."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    e = np.arange(len(src), dtype=np.int64)
    keep = src != dst
    I = np.concatenate([src[keep], dst[keep]])
    J = np.concatenate([dst[keep], src[keep]])
    E = np.concatenate([e[keep], e[keep]])
    return I, J, E


def starcheck(p: np.ndarray) -> np.ndarray:
    """Sec. 2.3 'Starcheck': s_i = (p_i = p_{p_i}); a vertex whose parent is not a
    root clears its own flag and its grandparent's; then s_i <- s_{p_i}."""
    n = len(p)
    s = np.ones(n, bool)
    pp = p[p]
    not_root_parent = p != pp
    s[not_root_parent] = False
    s[pp[not_root_parent]] = False
    s = np.where(s, s[p], s)
    return s


def multilinear(n, I, J, K, p, s):
    """Multilinear step: q_i = MinWeight_j f(p_i, a_ij, p_j) for i in a star, where
    f = (a_ij, p_j) if p_i != p_j else the identity.  Returns (q_key, q_parent)."""
    q_key = np.full(n, INF, np.uint64)
    q_par = np.full(n, -1, np.int64)
    out = (p[I] != p[J]) & s[I]
    np.minimum.at(q_key, I[out], K[out])
    # the least key of a row is one slot; its destination's parent rides along
    hit = out & (K == q_key[I])
    q_par[I[hit]] = p[J[hit]]
    return q_key, q_par


def project(n, q_key, q_par, p):
    """Projection: r_{p_i} = MinWeight_i q_i (projection onto the star root)."""
    r_key = np.full(n, INF, np.uint64)
    r_par = np.full(n, -1, np.int64)
    have = q_key != INF
    idx = np.nonzero(have)[0]
    np.minimum.at(r_key, p[idx], q_key[idx])
    hit = idx[q_key[idx] == r_key[p[idx]]]
    r_par[p[hit]] = q_par[hit]
    return r_key, r_par


def hook(p, r_key, r_par):
    """Hooking: p_i <- r_i^parent wherever r_i is not the identity."""
    p = p.copy()
    h = r_key != INF
    p[h] = r_par[h]
    return p


def tie_break(p, p_old, r_key):
    """Tie breaking and weight update: t_i = (i a star root, i < p_i, i = p_{p_i}); p_i <- i if t_i;
    every other root that hooked contributes its edge r_i to the forest."""
    n = len(p)
    i = np.arange(n)
    root = p_old == i
    t = root & (i < p) & (p[p] == i)
    p = np.where(t, i, p)
    add = root & (r_key != INF) & ~t
    edges = (r_key[add] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return p, t, edges


def csp_shortcut(p, p_prev):
    """Algorithm 3: changed = {(i, p_i) : p_i != p^prev_i}; every vertex then
    follows p_i through `changed` until p_i is not a key of it."""
    changed = {int(i): int(p[i]) for i in np.nonzero(p != p_prev)[0]}
    out = p.copy()
    for i in range(len(p)):
        x = int(out[i])
        steps = 0
        while x in changed:
            x = changed[x]
            steps += 1
            if steps > len(p):
                raise RuntimeError("cycle in the parent forest")
        out[i] = x
    return out


def shortcut_once(p, s):
    """One shortcut step (Algorithm 1, Sec. 2.3): every vertex outside a star
    takes its grandparent, all at once (reads the parents before the step)."""
    return np.where(s, p, p[p])


def as_msf(n: int, src, dst, w, wtype: int, max_rounds: int = 64, mode: str = "complete",
           stop_after: int = 0):
    """Runs Algorithm 2 to convergence.

    mode "complete": complete shortcutting by Algorithm 3 (Sec. 4.2) after every
    round, so every tree is a star when the next round starts.
    mode "original": the original schedule (Algorithm 1 and the printed
    Algorithm 2): starcheck, hooking of star roots only, tie breaking, then
    one shortcut step for the vertices outside a star (starcheck again).
    stop_after > 0 ends the loop after that many rounds (the partial forest).
    Returns dict(mask, labels, total, rounds, history=[p after each round],
    hooks=[#hooked roots per round], trees=[#trees with an outgoing edge])."""
    if mode not in ("complete", "original"):
        raise ValueError(mode)
    I, J, E = adjacency(n, src, dst)
    keys = edge_keys(w, wtype)
    K = keys[E]
    m = len(keys)
    p = np.arange(n, dtype=np.int64)                     # every vertex its own root
    p_old = np.full(n, -1, np.int64)                     # 'old' parent: none yet
    mask = np.zeros(m, np.uint8)
    history, hooks, trees = [], [], []
    rounds = 0
    while not np.array_equal(p, p_old):                  # loop test
        if stop_after and rounds == stop_after:
            break
        if rounds == max_rounds:
            raise RuntimeError("round limit")
        rounds += 1
        p_old = p.copy()                                 # remember p
        s = starcheck(p)
        q_key, q_par = multilinear(n, I, J, K, p, s)     # multilinear step
        r_key, r_par = project(n, q_key, q_par, p)       # projection
        trees.append(int(np.count_nonzero(r_key != INF)))
        p = hook(p, r_key, r_par)                        # hooking
        p, t, edges = tie_break(p, p_old, r_key)         # tie breaking, weight
        mask[edges] = 1
        hooks.append(int(len(edges)))
        if mode == "complete":
            p = csp_shortcut(p, p_old)                   # shortcut, complete
        else:
            p = shortcut_once(p, starcheck(p))           # shortcut, one step
        history.append(p.copy())
    # canonical labels: smallest vertex id per final tree
    lab = np.full(n, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(lab, p, np.arange(n))
    labels = lab[p].astype(np.int32)
    words = weight_words(w, wtype)
    wv = words.view(np.float32) if wtype == 0 else words
    total = exact_total(wv[mask.astype(bool)], wtype)
    return dict(mask=mask, labels=labels, total=total, rounds=rounds,
                history=history, hooks=hooks, trees=trees, parent=p)
