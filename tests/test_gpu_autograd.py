"""Differentiation of the forest weight (GPU): the backward kernel returns the
forest indicator times the incoming gradient, bit for bit, and agrees with
central finite differences where the weights are distinct."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import DEV, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_04865_gb300 import build_lib
    build_lib.build()


def test_backward_is_forest_indicator_single():
    import torch
    from paper_2110_04865_gb300 import api
    d = synth.workload("er4096")
    w = torch.from_numpy(d["w"]).to(DEV).requires_grad_(True)
    batch = api.Batch.single(d["n"], to_dev(d["src"]), to_dev(d["dst"]))
    totals, mask = api.msf_weight(w, batch)
    (3.0 * totals).sum().backward()
    omk, _, otot = oracle.kruskal(d["n"], d["src"], d["dst"], d["w"], 0)
    assert float(totals.item()) == otot
    assert np.array_equal(w.grad.cpu().numpy(), 3.0 * omk.astype(np.float32))


def test_backward_batched_scales_per_graph():
    import torch
    from paper_2110_04865_gb300 import api
    voff, eoff, s, d, w, _ = synth.batch(128, nmax=4096, seed=11)
    wt = torch.from_numpy(w).to(DEV).requires_grad_(True)
    batch = api.Batch(voff, eoff, to_dev(s), to_dev(d))
    totals, mask = api.msf_weight(wt, batch)
    gout = torch.arange(1, 129, dtype=torch.float64, device=DEV)
    (totals * gout).sum().backward()
    omk, _, otot = oracle.kruskal_batched(voff, eoff, s, d, w, 0)
    g_of_e = np.repeat(np.arange(128), np.diff(eoff))
    expect = omk.astype(np.float32) * (g_of_e + 1).astype(np.float32)
    assert np.array_equal(wt.grad.cpu().numpy(), expect)
    assert np.array_equal(totals.detach().cpu().numpy(), otot)


def test_finite_differences_distinct_weights():
    """Weights (pi(e)+1) 2^-k with k = ceil(log2(m+1)) and step h = 2^-(k+2):
    w +- h crosses no other weight and is exact in float32, and the sums are
    exact, so (W(w+h) - W(w-h)) / 2h equals the indicator exactly."""
    import torch
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(4)
    n, m = 3000, 12000
    s = rng.integers(0, n, m).astype(np.int32)
    d = rng.integers(0, n, m).astype(np.int32)
    k = int(np.ceil(np.log2(m + 1)))
    w = ((rng.permutation(m) + 1) * 2.0 ** -k).astype(np.float32)
    h = np.float32(2.0 ** -(k + 2))
    mk, _, _ = api.compute(n, to_dev(s), to_dev(d), to_dev(w))
    mk = mk.cpu().numpy()
    for e in rng.choice(m, 48, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        tp = float(api.compute(n, to_dev(s), to_dev(d), to_dev(wp))[2].cpu()[0])
        tm = float(api.compute(n, to_dev(s), to_dev(d), to_dev(wm))[2].cpu()[0])
        fd = (tp - tm) / (2 * float(h))
        assert fd == float(mk[e]), (e, fd, mk[e])


def test_finite_differences_batched_one_edge_per_graph():
    """Config-4 style batch with weights in (0,1): perturb one edge in every
    graph at once; only edges whose weight is unique within its graph are
    checked (at a tie the forest weight is not differentiable)."""
    from paper_2110_04865_gb300 import api
    G = 256
    voff, eoff, s, d, w, _ = synth.batch(G, nmax=8192, seed=21)
    h = np.float32(2.0 ** -24)   # weights are odd multiples of 2^-24: w +- h is exact, crosses none
    mk, _, _ = api.compute_batched(voff, eoff, to_dev(s), to_dev(d), to_dev(w))
    mk = mk.cpu().numpy()
    rng = np.random.default_rng(8)
    for trial in range(3):
        pick = np.array([rng.integers(eoff[g], eoff[g + 1]) if eoff[g + 1] > eoff[g] else -1 for g in range(G)])
        ok = pick >= 0
        for g in np.nonzero(ok)[0]:
            wg = w[eoff[g]:eoff[g + 1]]
            if np.count_nonzero(wg == w[pick[g]]) > 1 or s[pick[g]] == d[pick[g]]:
                ok[g] = False
        wp, wm = w.copy(), w.copy()
        wp[pick[ok]] += h
        wm[pick[ok]] -= h
        tp = api.compute_batched(voff, eoff, to_dev(s), to_dev(d), to_dev(wp))[2].cpu().numpy()
        tm = api.compute_batched(voff, eoff, to_dev(s), to_dev(d), to_dev(wm))[2].cpu().numpy()
        fd = (tp - tm) / (2 * float(h))
        for g in np.nonzero(ok)[0]:
            assert fd[g] == float(mk[pick[g]]), (g, fd[g], mk[pick[g]])


@pytest.fixture(scope="module")
def batch4096():
    """The 4096-graph batch (n log-uniform in [64, 65536], ER or 2-D random
    geometric, about 151 million edges) and the oracle's forests of it."""
    b = synth.workload("batch4096")
    omk, _, otot = oracle.kruskal_batched(b["voff"], b["eoff"], b["src"], b["dst"], b["w"], 0)
    return b, omk, otot


def test_backward_full_batch4096(batch4096):
    """Autograd on the whole 4096-graph batch: the totals are the oracle's and
    the gradient is the oracle's forest indicator times each graph's incoming
    gradient, bit for bit."""
    import torch
    from paper_2110_04865_gb300 import api
    b, omk, otot = batch4096
    G, eoff = b["G"], b["eoff"]
    wt = torch.from_numpy(b["w"]).to(DEV).requires_grad_(True)
    batch = api.Batch(b["voff"], eoff, to_dev(b["src"]), to_dev(b["dst"]))
    totals, mask = api.msf_weight(wt, batch)
    # per-graph gradients exactly representable in float32
    gout = (torch.arange(G, dtype=torch.float64, device=DEV) % 13 + 1) * 0.25
    (totals * gout).sum().backward()
    assert np.array_equal(totals.detach().cpu().numpy(), otot)
    assert np.array_equal(mask.cpu().numpy(), omk)
    g_of_e = np.repeat(np.arange(G), np.diff(eoff))
    expect = omk.astype(np.float32) * ((g_of_e % 13 + 1) * 0.25).astype(np.float32)
    assert np.array_equal(wt.grad.cpu().numpy(), expect)


def test_finite_differences_full_batch4096(batch4096):
    """Central differences on the whole batch: one edge per graph perturbed by
    h = 2^-24 (the weights are odd multiples of 2^-24, so w +- h is exact and
    crosses no other weight); checked where the edge's weight is unique in its
    graph (at a tie the forest weight is not differentiable)."""
    from paper_2110_04865_gb300 import api
    b, omk, _ = batch4096
    G, voff, eoff, s, d, w = b["G"], b["voff"], b["eoff"], b["src"], b["dst"], b["w"]
    h = np.float32(2.0 ** -24)
    ds, dd = to_dev(s), to_dev(d)
    rng = np.random.default_rng(12)
    checked = 0
    for _ in range(2):
        pick = np.array([rng.integers(eoff[g], eoff[g + 1]) if eoff[g + 1] > eoff[g] else -1 for g in range(G)])
        ok = pick >= 0
        for g in np.nonzero(ok)[0]:
            wg = w[eoff[g]:eoff[g + 1]]
            if np.count_nonzero(wg == w[pick[g]]) > 1 or s[pick[g]] == d[pick[g]]:
                ok[g] = False
        wp, wm = w.copy(), w.copy()
        wp[pick[ok]] += h
        wm[pick[ok]] -= h
        tp = api.compute_batched(voff, eoff, ds, dd, to_dev(wp))[2].cpu().numpy()
        tm = api.compute_batched(voff, eoff, ds, dd, to_dev(wm))[2].cpu().numpy()
        fd = (tp - tm) / (2 * float(h))
        sel = np.nonzero(ok)[0]
        assert np.array_equal(fd[sel], omk[pick[sel]].astype(np.float64))
        checked += len(sel)
    assert checked > 4000
