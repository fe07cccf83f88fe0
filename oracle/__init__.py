"""ORACLE: test infrastructure only.

Plain, slow, obviously correct CPU implementations of what the library
computes.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import this package; the library never does, and nothing here shares code
with it.

Contents
  * ``kruskal`` / ``kruskal_mt`` / ``kruskal_batched`` (``kruskal.c``): the unique minimum
    spanning forest under the strict order (ord(w), edge id) -- the plain
    definition the method reaches (Sec. 1, Sec. 2.3).  Returns the edge mask over
    the input COO entries, canonical component labels (smallest vertex id of
    each component) and the exact total weight.
  * ``exact_total``: the forest weight, summed exactly and rounded once to
    double (math.fsum is Shewchuk's correctly rounded float summation).
  * ``prim`` (prim.py), ``brute_force`` (brute.py): independent forests used
    only to pin Kruskal.
  * ``as_rounds`` (as_rounds.py): Algorithm 2 (algebraic Awerbuch-Shiloach)
    with complete shortcutting (Sec. 4.2, Algorithm 3), step by step in the
    paper's order and notation, for per-step checks of the GPU kernels.

Readings of the paper used here (the paper assumes distinct weights):
  ties are broken by the input COO index of the undirected edge; float32
  weights are ordered by their value with -0 == +0; NaN is invalid.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile kruskal.c into _build/liboracle.so with gcc (OpenMP when
    available, for the all-cores variant's sort)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "kruskal.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_kruskal.restype = ctypes.c_int64
            lib.oracle_kruskal.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 3 + \
                [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_kruskal_mt.restype = ctypes.c_int64
            lib.oracle_kruskal_mt.argtypes = lib.oracle_kruskal.argtypes + [ctypes.c_int]
            _lib = lib
    return _lib


def weight_words(w: np.ndarray, wtype: int) -> np.ndarray:
    """Raw 32-bit words of a float32 (wtype 0) or uint32 (wtype 1) weight array."""
    w = np.ascontiguousarray(w)
    if wtype == 0:
        return w.astype(np.float32, copy=False).view(np.uint32)
    return w.astype(np.uint32, copy=False)


def ord_words(words: np.ndarray, wtype: int) -> np.ndarray:
    """Order-preserving map of weight words to uint32 (numpy restatement of the
    one in kruskal.c, for the per-step oracle and the tests)."""
    b = np.asarray(words, dtype=np.uint32)
    if wtype != 0:
        return b.copy()
    b = np.where(b == np.uint32(0x80000000), np.uint32(0), b)
    neg = (b >> np.uint32(31)) != 0
    return np.where(neg, ~b, b ^ np.uint32(0x80000000)).astype(np.uint32)


def edge_keys(w: np.ndarray, wtype: int) -> np.ndarray:
    """key(e) = ord(w_e) * 2^32 + e as uint64 (the strict total edge order)."""
    o = ord_words(weight_words(w, wtype), wtype).astype(np.uint64)
    return (o << np.uint64(32)) | np.arange(len(o), dtype=np.uint64)


def exact_total(w_selected: np.ndarray, wtype: int) -> float:
    """Exact sum of the selected weights, rounded once to the nearest double."""
    if wtype != 0:
        # fewer than 2^31 forest edges of at most 2^32-1 each: no uint64 overflow
        return float(int(np.asarray(w_selected, dtype=np.uint64).sum(dtype=np.uint64)))
    v = np.asarray(w_selected, dtype=np.float32).astype(np.float64)
    pos_inf = bool(np.any(v == np.inf))
    neg_inf = bool(np.any(v == -np.inf))
    if pos_inf and neg_inf:
        return float("nan")
    if pos_inf:
        return float("inf")
    if neg_inf:
        return float("-inf")
    return math.fsum(v.tolist())


def kruskal(n: int, src, dst, w, wtype: int, threads: int = 0):
    """Minimum spanning forest of one graph -> (mask uint8[m], labels int32[n], total).
    threads > 0: the keys are built and sorted on that many threads (the same
    forest; a CPU baseline on all cores), the union-find scan stays sequential."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    words = np.ascontiguousarray(weight_words(w, wtype))
    m = len(src)
    if wtype == 0 and np.isnan(words.view(np.float32)).any():
        raise ValueError("NaN weight")
    if m and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("vertex index out of range")
    mask = np.zeros(m, np.uint8)
    labels = np.zeros(n, np.int32)
    if threads > 0:
        got = _load().oracle_kruskal_mt(n, m, src.ctypes.data, dst.ctypes.data, words.ctypes.data,
                                        wtype, mask.ctypes.data, labels.ctypes.data, threads)
    else:
        got = _load().oracle_kruskal(n, m, src.ctypes.data, dst.ctypes.data, words.ctypes.data,
                                     wtype, mask.ctypes.data, labels.ctypes.data)
    if got < 0:
        raise MemoryError("oracle allocation failed")
    wv = words.view(np.float32) if wtype == 0 else words
    return mask, labels, exact_total(wv[mask.astype(bool)], wtype)


def kruskal_mt(n: int, src, dst, w, wtype: int, threads: int):
    """kruskal() with the key construction and sort on `threads` threads."""
    return kruskal(n, src, dst, w, wtype, threads=max(int(threads), 1))


def kruskal_batched(voff, eoff, src, dst, w, wtype: int):
    """Per-graph forests of a batch with LOCAL vertex ids.
    Returns (mask uint8[sum m], labels int32[sum n] (local), totals float64[G])."""
    voff = np.asarray(voff, np.int64)
    eoff = np.asarray(eoff, np.int64)
    G = len(voff) - 1
    mask = np.zeros(int(eoff[-1]), np.uint8)
    labels = np.zeros(int(voff[-1]), np.int32)
    totals = np.zeros(G, np.float64)
    for g in range(G):
        a, b = int(eoff[g]), int(eoff[g + 1])
        mk, lb, tot = kruskal(int(voff[g + 1] - voff[g]), src[a:b], dst[a:b], w[a:b], wtype)
        mask[a:b] = mk
        labels[int(voff[g]):int(voff[g + 1])] = lb
        totals[g] = tot
    return mask, labels, totals
