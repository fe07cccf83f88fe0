"""Helpers shared by the GPU tests: run the library through its C ABI on
cuda:0 and compare with the oracle."""
from __future__ import annotations

import math

import numpy as np

DEV = "cuda:0"


def to_dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(DEV)


def run_single(n, src, dst, w, host=False):
    from paper_2110_04865_gb300 import api
    if host:
        w_in = np.ascontiguousarray(w.view(np.int32) if w.dtype == np.uint32 else w)
        mk, lb, tt = api.compute(n, np.ascontiguousarray(src), np.ascontiguousarray(dst), w_in)
        return mk, lb, float(tt[0])
    mk, lb, tt = api.compute(n, to_dev(src), to_dev(dst), to_dev(w))
    return mk.cpu().numpy(), lb.cpu().numpy(), float(tt.cpu()[0])


def same_total(a: float, b: float) -> bool:
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return a == b


def assert_parity(n, src, dst, w, wtype, got=None, host=False):
    import oracle
    mk, lb, tot = got if got is not None else run_single(n, src, dst, w, host=host)
    omk, olb, otot = oracle.kruskal(n, src, dst, w, wtype)
    assert mk.dtype == np.uint8 and lb.dtype == np.int32
    bad = np.nonzero(mk != omk)[0]
    assert len(bad) == 0, f"{len(bad)} mask entries differ, first {bad[:5]}"
    badl = np.nonzero(lb != olb)[0]
    assert len(badl) == 0, f"{len(badl)} labels differ, first {badl[:5]}"
    assert same_total(tot, otot), (tot, otot)
    return omk, olb, otot
