"""Seeded synthetic graph workloads (inputs only).

The generators live in ``gen.c`` (compiled on first use with gcc); this module
wraps them with numpy.  Nothing here computes any part of the minimum spanning
forest: it produces COO edge lists ``(src, dst, w)`` and, for batches, vertex
and edge offsets.  Weights are returned as numpy float32 (``wtype=0``) or
uint32 (``wtype=1``) arrays.

Workloads (seed 20211010 + workload number unless given):
  * ``er(n, m)``            uniform random multigraph (self-loops, duplicates kept)
  * ``rmat(scale, ef)``     R-MAT a,b,c,d = .57,.19,.19,.05, ef * 2^scale draws
  * ``grid3d(nx, ny, nz)``  7-point lattice, u32 weights in [1,1000] by default
  * ``rgg(n, deg)``         2-D random geometric graph with average degree deg
  * ``batch(G)``            G graphs, n log-uniform in [64, 65536], ER or RGG
  * ``rmat<scale>p``        R-MAT with vertex ids permuted by a fixed bijection
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

BASE_SEED = 20211010
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile gen.c into _build/libsynth.so (OpenMP when available)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", tmp, "-lm"]
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
            lib.synth_draw.restype = _u64
            lib.synth_draw.argtypes = [_u64, _u64, _u64]
            lib.synth_er.argtypes = [_i64, _i64, _u64, ctypes.c_int, _ptr, _ptr, _ptr]
            lib.synth_rmat.argtypes = [ctypes.c_int, _i64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _u64, ctypes.c_int, _ptr, _ptr, _ptr]
            lib.synth_grid3d_count.restype = _i64
            lib.synth_grid3d_count.argtypes = [_i64, _i64, _i64]
            lib.synth_grid3d.argtypes = [_i64, _i64, _i64, _u64, ctypes.c_int, _ptr, _ptr, _ptr]
            lib.synth_rgg_count.restype = _i64
            lib.synth_rgg_count.argtypes = [_i64, ctypes.c_double, _u64]
            lib.synth_rgg.argtypes = [_i64, ctypes.c_double, _u64, ctypes.c_int, _ptr, _ptr, _ptr]
            lib.synth_batch_sizes.argtypes = [_i64, _i64, _i64, ctypes.c_double, _u64,
                                              _ptr, _ptr, _ptr]
            lib.synth_batch_fill.argtypes = [_i64, ctypes.c_double, _u64, ctypes.c_int,
                                             _ptr, _ptr, _ptr, _ptr, _ptr, _ptr]
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _alloc(m: int, wtype: int):
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    w = np.empty(m, np.uint32)
    return src, dst, w


def _wview(w: np.ndarray, wtype: int) -> np.ndarray:
    return w.view(np.float32) if wtype == 0 else w


def draw(seed: int, stream: int, i: int) -> int:
    """One counter-based splitmix64 value (for tests of the generator)."""
    return int(_load().synth_draw(seed, stream, i))


def er(n: int, m: int, seed: int = BASE_SEED + 1, wtype: int = 0):
    src, dst, w = _alloc(m, wtype)
    _load().synth_er(n, m, seed, wtype, _p(src), _p(dst), _p(w))
    return src, dst, _wview(w, wtype)


def rmat(scale: int, edge_factor: int = 16, seed: int = BASE_SEED + 2, wtype: int = 0,
         a: float = 0.57, b: float = 0.19, c: float = 0.19):
    m = edge_factor << scale
    src, dst, w = _alloc(m, wtype)
    _load().synth_rmat(scale, m, a, b, c, seed, wtype, _p(src), _p(dst), _p(w))
    return src, dst, _wview(w, wtype)


def grid3d_count(nx: int, ny: int, nz: int) -> int:
    return int(_load().synth_grid3d_count(nx, ny, nz))


def grid3d(nx: int, ny: int, nz: int, seed: int = BASE_SEED + 3, wtype: int = 1):
    m = grid3d_count(nx, ny, nz)
    src, dst, w = _alloc(m, wtype)
    _load().synth_grid3d(nx, ny, nz, seed, wtype, _p(src), _p(dst), _p(w))
    return src, dst, _wview(w, wtype)


def rgg(n: int, deg: float = 8.0, seed: int = BASE_SEED + 4, wtype: int = 0):
    lib = _load()
    m = int(lib.synth_rgg_count(n, deg, seed))
    src, dst, w = _alloc(m, wtype)
    lib.synth_rgg(n, deg, seed, wtype, _p(src), _p(dst), _p(w))
    return src, dst, _wview(w, wtype)


def batch(G: int, nmin: int = 64, nmax: int = 65536, deg: float = 8.0,
          seed: int = BASE_SEED + 4, wtype: int = 0):
    """Returns (voff[G+1], eoff[G+1], src, dst, w, kind) with LOCAL vertex ids."""
    lib = _load()
    nv = np.empty(G, np.int64)
    ne = np.empty(G, np.int64)
    kind = np.empty(G, np.int32)
    lib.synth_batch_sizes(G, nmin, nmax, deg, seed, _p(nv), _p(ne), _p(kind))
    voff = np.zeros(G + 1, np.int64)
    eoff = np.zeros(G + 1, np.int64)
    np.cumsum(nv, out=voff[1:])
    np.cumsum(ne, out=eoff[1:])
    src, dst, w = _alloc(int(eoff[-1]), wtype)
    lib.synth_batch_fill(G, deg, seed, wtype, _p(nv), _p(eoff), _p(kind),
                         _p(src), _p(dst), _p(w))
    return voff, eoff, src, dst, _wview(w, wtype), kind


def permutation(bits: int) -> np.ndarray:
    """A fixed bijection of [0, 2^bits) (xorshift-multiply rounds, each
    invertible modulo 2^bits), as an int32 lookup table."""
    mask = np.uint64((1 << bits) - 1)
    x = np.arange(1 << bits, dtype=np.uint64) ^ (np.uint64(0x5BD1E995) & mask)
    for mul in (0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9, 0x94D049BB133111EB):
        x ^= x >> np.uint64(max(bits // 2, 1))
        x = (x * np.uint64(mul | 1)) & mask
    return x.astype(np.int32)


# The five workloads, by what they are.
def workload(name: str):
    """Named workloads.  Returns dict(n, src, dst, w, wtype) or a batch dict."""
    if name == "er4096":
        s, d, w = er(4096, 32768, BASE_SEED + 1, 0)
        return dict(n=4096, src=s, dst=d, w=w, wtype=0)
    if name == "er20":
        # uniform random graph with R-MAT 20's sizes (no hubs)
        s, d, w = er(1 << 20, 16 << 20, BASE_SEED + 6, 0)
        return dict(n=1 << 20, src=s, dst=d, w=w, wtype=0)
    if name.startswith("rmat") and name.endswith("p"):
        # rmat<scale>p: the same graph with vertex ids permuted (hubs no longer
        # at low ids)
        d = workload(name[:-1])
        scale = int(name[4:-1].split("e")[0])
        perm = permutation(scale)
        d["src"] = perm[d["src"]]
        d["dst"] = perm[d["dst"]]
        return d
    if name.startswith("rmat"):
        # rmat<scale> (edge factor 16) or rmat<scale>e<edge factor>
        body = name[4:]
        scale, ef = (int(body.split("e")[0]), int(body.split("e")[1])) if "e" in body else (int(body), 16)
        s, d, w = rmat(scale, ef, BASE_SEED + (2 if scale < 26 else 5), 0)
        return dict(n=1 << scale, src=s, dst=d, w=w, wtype=0)
    if name.startswith("grid"):
        k = int(name[4:])
        s, d, w = grid3d(k, k, k, BASE_SEED + 3, 1)
        return dict(n=k * k * k, src=s, dst=d, w=w, wtype=1)
    if name.startswith("batch"):
        G = int(name[5:])
        voff, eoff, s, d, w, kind = batch(G, seed=BASE_SEED + 4)
        return dict(G=G, voff=voff, eoff=eoff, src=s, dst=d, w=w, wtype=0, kind=kind)
    raise KeyError(name)


def log_uniform_mean(nmin: int = 64, nmax: int = 65536) -> float:
    return (nmax - nmin) / math.log(nmax / nmin)
