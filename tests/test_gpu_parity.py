"""GPU path vs the CPU oracle, element by element, through the C ABI.

Edge masks and labels must match bit for bit and the totals exactly (the
forest is unique under the (weight, edge id) order and both sides sum
exactly, then round once).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from golden_io import all_fixtures
from gpu_util import DEV, assert_parity, run_single, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_04865_gb300 import _abi, build_lib
    build_lib.build()
    _abi.load()
    yield


def rand_graph(rng, n, m, wtype, levels=None, negative=False):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if wtype == 0:
        if levels:
            w = rng.choice(np.linspace(-1 if negative else 0.0625, 1, levels), m).astype(np.float32)
        else:
            w = rng.random(m).astype(np.float32) - np.float32(0.5 if negative else 0)
    else:
        w = rng.integers(1, (levels or 1000) + 1, m).astype(np.uint32)
    return src, dst, w


@pytest.mark.parametrize("seed", range(24))
def test_random_small_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 6 * n))
    wtype = seed % 2
    src, dst, w = rand_graph(rng, n, m, wtype, levels=[None, 3, 50][seed % 3], negative=(seed % 4 == 1))
    assert_parity(n, src, dst, w, wtype)


@pytest.mark.parametrize("fx", all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixtures(fx):
    mk, lb, tot = run_single(fx["n"], fx["src"], fx["dst"], fx["w"])
    assert np.array_equal(mk, fx["mask"])
    assert np.array_equal(lb, fx["labels"])
    assert tot == fx["total"]


def test_edge_cases():
    e = np.zeros(0, np.int32)
    # no edges
    for n in (1, 7):
        mk, lb, tot = run_single(n, e, e, np.zeros(0, np.float32))
        assert len(mk) == 0 and list(lb) == list(range(n)) and tot == 0.0
    # only self-loops
    s = np.arange(10, dtype=np.int32)
    assert_parity(10, s, s, np.ones(10, np.float32), 0)
    # a star around vertex 0 (one very long row)
    rng = np.random.default_rng(1)
    n = 20000
    leaves = np.arange(1, n, dtype=np.int32)
    assert_parity(n, np.zeros(n - 1, np.int32), leaves, rng.random(n - 1).astype(np.float32), 0)
    # paths: increasing weights hook into one long chain (deep pointer jumping)
    n = 200000
    a, b = np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)
    assert_parity(n, a, b, np.arange(1, n, dtype=np.uint32), 1)
    assert_parity(n, a, b, np.arange(n - 1, 0, -1, dtype=np.uint32), 1)
    # complete graph, equal weights: ids decide every tie
    iu, ju = np.triu_indices(300, 1)
    assert_parity(300, iu.astype(np.int32), ju.astype(np.int32), np.full(len(iu), 5, np.uint32), 1)
    # signed zeros, infinities, negatives, duplicates
    src = rng.integers(0, 50, 400).astype(np.int32)
    dst = rng.integers(0, 50, 400).astype(np.int32)
    w = rng.choice(np.array([-0.0, 0.0, -1.5, 2.0, np.inf, -np.inf, 1e-30, -3e38], np.float32), 400)
    assert_parity(50, src, dst, w, 0)


def test_er_4096():
    d = synth.workload("er4096")
    assert_parity(d["n"], d["src"], d["dst"], d["w"], 0)


@pytest.mark.parametrize("scale", [12, 16, 20])
def test_rmat(scale):
    d = synth.workload(f"rmat{scale}")
    assert_parity(d["n"], d["src"], d["dst"], d["w"], 0)


@pytest.mark.parametrize("k", [16, 64, 256])
def test_grid3d(k):
    d = synth.workload(f"grid{k}")
    assert_parity(d["n"], d["src"], d["dst"], d["w"], 1)


def test_compaction_and_tile_shapes_do_not_change_results():
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload("rmat16")
    ref = None
    opts = (_abi.OPT_COMPACT_TAU, _abi.OPT_SLOTS_PER_LANE, _abi.OPT_PREFETCH, _abi.OPT_EXEC_MODE,
            _abi.OPT_BLOCKS_PER_SM)
    old = {o: _abi.msf_get_option(o) for o in opts}
    cases = [(tau, spl, pf, ex, bps) for tau in (0.0, 0.3, 0.9) for spl in (4, 8, 16) for pf in (0, 1)
             for ex, bps in ((0, 4), (1, 2))]
    try:
        for tau, spl, pf, ex, bps in cases:
            for o, v in zip(opts, (tau, spl, pf, ex, bps)):
                _abi.msf_set_option(o, v)
            g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
            mk, lb, tt = g.compute()
            st = g.stats()
            g.free()
            got = (mk.cpu().numpy(), lb.cpu().numpy(), float(tt.cpu()[0]))
            if tau == 0.9:
                assert st.compactions > 0
            if tau == 0.0:
                assert st.compactions == 0
            if ref is None:
                ref = assert_parity(d["n"], d["src"], d["dst"], d["w"], 0, got=got)
            else:
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
                assert got[2] == ref[2]
    finally:
        for o, v in old.items():
            _abi.msf_set_option(o, v)


def test_grid_with_compaction_and_host_loop():
    from paper_2110_04865_gb300 import _abi
    d = synth.workload("grid64")
    old = {o: _abi.msf_get_option(o) for o in (_abi.OPT_COMPACT_TAU, _abi.OPT_EXEC_MODE)}
    try:
        for tau, ex in ((0.9, 0), (0.9, 1), (0.5, 1)):
            _abi.msf_set_option(_abi.OPT_COMPACT_TAU, tau)
            _abi.msf_set_option(_abi.OPT_EXEC_MODE, ex)
            assert_parity(d["n"], d["src"], d["dst"], d["w"], 1)
    finally:
        for o, v in old.items():
            _abi.msf_set_option(o, v)


def test_repeat_compute_and_host_buffers():
    from paper_2110_04865_gb300 import api
    d = synth.workload("rmat12")
    g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    first = [x.cpu().numpy() for x in g.compute()]
    second = [x.cpu().numpy() for x in g.compute()]
    g.free()
    for a, b in zip(first, second):
        assert np.array_equal(a, b)
    # host (numpy) inputs and outputs are staged by the library
    assert_parity(d["n"], d["src"], d["dst"], d["w"], 0, host=True)


def test_rounds_are_logarithmic():
    from paper_2110_04865_gb300 import api
    d = synth.workload("grid64")
    g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    g.compute()
    st = g.stats()
    g.free()
    # complete shortcutting: every tree with an outgoing edge hooks or is
    # hooked onto, so trees with outgoing edges at least halve per round
    assert 1 <= st.rounds <= int(np.ceil(np.log2(d["n"]))) + 2
    assert st.forest_edges == d["n"] - 1


def test_csr_input_form():
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(5)
    n, m = 3000, 12000
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    keep = u != v
    u, v = u[keep], v[keep]
    w = (rng.integers(1, 200, len(u))).astype(np.float32)
    # symmetric CSR: both directions, rows sorted, arbitrary order inside a row
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    order = np.argsort(rows, kind="stable")
    rows, cols, ww = rows[order], cols[order], ww[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    g = api.Graph(n, None, to_dev(cols.astype(np.int32)), to_dev(ww), row_ptr=to_dev(row_ptr))
    mk, lb, tt = g.compute()
    g.free()
    # the definition applied to the slots with row < column (edge id = slot)
    src_slots = np.where(rows < cols, rows, cols).astype(np.int32)
    omk, olb, otot = oracle.kruskal(n, src_slots, cols.astype(np.int32), ww, 0)
    assert np.array_equal(mk.cpu().numpy(), omk)
    assert np.array_equal(lb.cpu().numpy(), olb)
    assert float(tt.cpu()[0]) == otot


def test_min_edge_kernel_matches_definition():
    """One multilinear application with projection (Sec. 3.1, Algorithm 2
    multilinear and projection steps) on a random star forest, against the per-step oracle."""
    import torch
    from oracle import as_rounds
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(9)
    for n, m, roots in [(2000, 9000, 37), (50000, 400000, 5000), (5, 12, 5)]:
        src, dst, w = rand_graph(rng, n, m, 0, levels=40)
        root_ids = rng.choice(n, roots, replace=False)
        p = root_ids[rng.integers(0, roots, n)]
        p[root_ids] = root_ids
        g = api.Graph(n, to_dev(src), to_dev(dst), to_dev(w))
        r = g.min_edge(torch.from_numpy(p.astype(np.int32)).to(DEV))
        g.free()
        I, J, E = as_rounds.adjacency(n, src, dst)
        K = oracle.edge_keys(w, 0)[E]
        q_key, q_par = as_rounds.multilinear(n, I, J, K, p.astype(np.int64), np.ones(n, bool))
        r_key, r_par = as_rounds.project(n, q_key, q_par, p.astype(np.int64))
        assert np.array_equal(r.cpu().numpy().view(np.uint64), r_key)


@pytest.mark.parametrize("G,nmax", [(1, 2000), (64, 4096), (4096, 65536)])
def test_batched(G, nmax):
    from paper_2110_04865_gb300 import api
    voff, eoff, s, d, w, kind = synth.batch(G, nmax=nmax, seed=77 + G)
    mk, lb, tt = api.compute_batched(voff, eoff, to_dev(s), to_dev(d), to_dev(w))
    omk, olb, otot = oracle.kruskal_batched(voff, eoff, s, d, w, 0)
    assert np.array_equal(mk.cpu().numpy(), omk)
    assert np.array_equal(lb.cpu().numpy(), olb)
    assert np.array_equal(tt.cpu().numpy(), otot)


def test_batched_with_empty_graphs_and_u32():
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(3)
    nv = [5, 0, 1, 40, 3]
    ne = [6, 0, 0, 100, 0]
    voff = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
    src = np.concatenate([rng.integers(0, max(a, 1), b) for a, b in zip(nv, ne)]).astype(np.int32)
    dst = np.concatenate([rng.integers(0, max(a, 1), b) for a, b in zip(nv, ne)]).astype(np.int32)
    w = rng.integers(1, 4, len(src)).astype(np.uint32)
    mk, lb, tt = api.compute_batched(voff, eoff, to_dev(src), to_dev(dst), to_dev(w))
    omk, olb, otot = oracle.kruskal_batched(voff, eoff, src, dst, w, 1)
    assert np.array_equal(mk.cpu().numpy(), omk)
    assert np.array_equal(lb.cpu().numpy(), olb)
    assert np.array_equal(tt.cpu().numpy(), otot)


@pytest.mark.parametrize("build", [0, 1, 2, 3])
def test_batched_offsets_on_block_boundaries(build):
    """A batch whose vertex and edge offsets fall on and next to multiples of
    4096 (the width of the blocks of the offset tables that locate an id's
    graph), with runs of empty graphs there and graphs spanning several
    blocks, through every builder."""
    from paper_2110_04865_gb300 import _abi, api
    rng = np.random.default_rng(4096 + build)
    nv = [4096, 0, 0, 1, 4095, 0, 12293, 2, 0, 4096, 1, 0]
    ne = [4096, 0, 0, 0, 8191, 0, 20000, 1, 0, 4095, 0, 0]
    voff = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
    src = np.concatenate([rng.integers(0, max(a, 1), b) for a, b in zip(nv, ne)]).astype(np.int32)
    dst = np.concatenate([rng.integers(0, max(a, 1), b) for a, b in zip(nv, ne)]).astype(np.int32)
    w = rng.integers(1, 50, len(src)).astype(np.uint32)
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, build)
        mk, lb, tt = api.compute_batched(voff, eoff, to_dev(src), to_dev(dst), to_dev(w))
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)
    omk, olb, otot = oracle.kruskal_batched(voff, eoff, src, dst, w, 1)
    assert np.array_equal(mk.cpu().numpy(), omk)
    assert np.array_equal(lb.cpu().numpy(), olb)
    assert np.array_equal(tt.cpu().numpy(), otot)


def test_mask_written_at_every_alignment():
    """The edge mask through a caller pointer at every offset modulo 16
    (the full compute writes the whole mask from the forest's bitmap, with
    16-byte stores between an unaligned head and tail): equal to the
    oracle's, and no byte outside it touched."""
    import torch
    from paper_2110_04865_gb300 import _abi
    rng = np.random.default_rng(16)
    cases = [synth.workload("er4096")]
    for n, m in ((6, 7), (20, 37)):
        s_, d_, w_ = rand_graph(rng, n, m, 0, levels=5)
        cases.append({"n": n, "src": s_, "dst": d_, "w": w_, "wtype": 0})
    sh = torch.cuda.current_stream().cuda_stream
    for d in cases:
        n, m = d["n"], len(d["src"])
        omk, olb, otot = oracle.kruskal(n, d["src"], d["dst"], d["w"], d["wtype"])
        src, dst, w = to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"])
        buf = torch.empty(m + 48, dtype=torch.uint8, device=DEV)
        lb = torch.empty(n, dtype=torch.int32, device=DEV)
        tt = torch.empty(1, dtype=torch.float64, device=DEV)
        for off in range(16):
            buf.fill_(7)
            g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), d["wtype"], 0, sh)
            _abi.msf_compute(g, buf.data_ptr() + off, lb.data_ptr(), tt.data_ptr(), sh)
            _abi.msf_free(g)
            got = buf.cpu().numpy()
            assert np.array_equal(got[off:off + m], omk), (m, off)
            assert np.all(got[:off] == 7) and np.all(got[off + m:] == 7), (m, off)
            assert np.array_equal(lb.cpu().numpy(), olb)
            assert float(tt.cpu()[0]) == otot


def test_host_inputs_read_in_place():
    """With MSF_OPT_HOST_INPUT = 1, page-locked host edge arrays are read by
    the build kernels in place; pageable ones are still copied.  Same forest."""
    import torch
    from paper_2110_04865_gb300 import _abi, api
    old = _abi.msf_get_option(_abi.OPT_HOST_INPUT)
    try:
        _abi.msf_set_option(_abi.OPT_HOST_INPUT, 1)
        for wl in ("rmat16", "grid16", "er4096"):
            d = synth.workload(wl)
            wv = d["w"].view(np.int32) if d["w"].dtype == np.uint32 else d["w"]
            hs = torch.from_numpy(np.ascontiguousarray(d["src"])).pin_memory()
            hd = torch.from_numpy(np.ascontiguousarray(d["dst"])).pin_memory()
            hw = torch.from_numpy(np.ascontiguousarray(wv)).pin_memory()
            mk, lb, tt = api.compute(d["n"], hs.numpy(), hd.numpy(), hw.numpy())
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"], got=(mk, lb, float(tt[0])))
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"], host=True)  # pageable
    finally:
        _abi.msf_set_option(_abi.OPT_HOST_INPUT, old)


@pytest.mark.parametrize("build", [0, 1, 2, 3])
def test_invalid_inputs_are_rejected(build):
    """Out-of-range vertices and NaN weights are rejected by every builder's
    validation (the bucketed builder validates inside its first pass)."""
    from paper_2110_04865_gb300 import MsfError, _abi, api
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, build)
        s = np.array([0, 1, 2], np.int32)
        d = np.array([1, 2, 3], np.int32)
        with pytest.raises(MsfError) as ei:
            api.compute(3, to_dev(s), to_dev(d), to_dev(np.ones(3, np.float32)))
        assert ei.value.code == 1
        with pytest.raises(MsfError) as ei:
            api.compute(4, to_dev(s), to_dev(d), to_dev(np.array([1, np.nan, 2], np.float32)))
        assert ei.value.code == 1
        # a large edge list with one bad vertex in the middle (16-byte loads)
        rng = np.random.default_rng(5)
        bs, bd, bw = rand_graph(rng, 5000, 100003, 0)
        bd[50001] = 5000
        with pytest.raises(MsfError) as ei:
            api.compute(5000, to_dev(bs), to_dev(bd), to_dev(bw))
        assert ei.value.code == 1
        # one NaN weight in the middle of a large list (the bucketed builder
        # checks weights in its scatter), and on more than 2^22 vertices
        for nv in (5000, (1 << 22) + 77):
            bs, bd, bw = rand_graph(rng, nv, 100003, 0)
            bw[70001] = np.nan
            with pytest.raises(MsfError) as ei:
                api.compute(nv, to_dev(bs), to_dev(bd), to_dev(bw))
            assert ei.value.code == 1 and "NaN" in str(ei.value)
        # the library stays usable
        assert_parity(4, s, d, np.array([3, 1, 2], np.float32), 0)
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


def test_limits_return_errors_without_hanging():
    """The round loop and pointer jumping are bounded; running out of either
    returns a status (the GPU is not hung and stays usable).  The path's
    hook chain (depth n - 1) cannot settle in one shortcut pass: a pass moves
    a changed root at most 16 hops (plus whatever concurrent updates show it)."""
    from paper_2110_04865_gb300 import MsfError, _abi, api
    n = 1 << 16
    a, b = np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)
    w = np.arange(1, n, dtype=np.uint32)
    old_r = _abi.msf_get_option(_abi.OPT_ROUND_LIMIT)
    old_j = _abi.msf_get_option(_abi.OPT_JUMP_LIMIT)
    try:
        _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, 1)
        rng = np.random.default_rng(0)
        s, d, ww = rand_graph(rng, 1000, 3000, 0)
        with pytest.raises(MsfError) as ei:
            api.compute(1000, to_dev(s), to_dev(d), to_dev(ww))
        assert ei.value.code == 4
        _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, old_r)
        _abi.msf_set_option(_abi.OPT_JUMP_LIMIT, 1)
        with pytest.raises(MsfError) as ei:
            api.compute(n, to_dev(a), to_dev(b), to_dev(w))
        assert ei.value.code == 5
    finally:
        _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, old_r)
        _abi.msf_set_option(_abi.OPT_JUMP_LIMIT, old_j)
    assert_parity(n, a, b, w, 1)


def _path(weights):
    w = np.asarray(weights)
    k = len(w)
    return k + 1, np.arange(k, dtype=np.int32), np.arange(1, k + 1, dtype=np.int32), w


@pytest.mark.parametrize("case", [
    [1.0, 2.0 ** -53],                       # exact tie: stays at 1
    [1.0, 2.0 ** -53, 2.0 ** -100],          # just above the tie: rounds up
    [1.0 + 2.0 ** -23, 2.0 ** -53],          # tie with an even neighbour
    [1.0, 2.0 ** -53, 2.0 ** -54],           # three quarters of an ulp
    [1.0, -(2.0 ** -54)],                    # tie below 1
    [2.0 ** 100, 1.0, -(2.0 ** 100)],        # cancellation
    [2.0 ** -149, 2.0 ** -149, -(2.0 ** -148), 2.0 ** -126],  # subnormals
    [-(2.0 ** 127), -(2.0 ** 127), 2.0 ** -149],
])
def test_exact_totals_rounding(case):
    """A path keeps every edge, so the total is the exact sum of all weights,
    rounded once (compared with the oracle's math.fsum)."""
    n, s, d, w = _path(np.array(case, np.float32))
    assert_parity(n, s, d, w, 0)


def test_exact_totals_random_exponents_and_u32_rounding():
    rng = np.random.default_rng(17)
    for _ in range(5):
        k = 3000
        mant = rng.integers(1, 1 << 24, k).astype(np.float64)
        expo = rng.integers(-149, 104, k)
        w = (rng.choice([-1.0, 1.0], k) * mant * np.exp2(expo.astype(np.float64))).astype(np.float32)
        w = w[np.isfinite(w)]
        n, s, d, w = _path(w)
        assert_parity(n, s, d, w, 0)
    # uint32: a sum above 2^53 that is odd rounds to even
    k = (1 << 22) + 1
    w = np.full(k, 0xFFFFFFFF, np.uint32)
    w[-1] = 1
    n, s, d, w = _path(w)
    assert_parity(n, s, d, w, 1)


SCHEDULES = {0: "complete", 1: "original", 2: "complete", 3: "complete"}


def expected_rounds(ref, mode, early_stop=True):
    """Rounds the device loop runs: the oracle's, or -- with early stop and a
    complete schedule -- the first round after which at most one tree with an
    outgoing edge is left."""
    if early_stop and SCHEDULES[mode] == "complete":
        for i, (t, h) in enumerate(zip(ref["trees"], ref["hooks"])):
            if h > 0 and t <= h + 1:
                return i + 1
    return ref["rounds"]


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("workload", ["rmat12", "grid16", "er4096"])
def test_shortcut_schedules(mode, workload):
    """Every schedule gives the oracle's forest, with the oracle's round count
    (the complete schedules share one trajectory; the original one its own)."""
    from oracle import as_rounds
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload(workload)
    old = {o: _abi.msf_get_option(o) for o in (_abi.OPT_SHORTCUT, _abi.OPT_OS_THRESHOLD, _abi.OPT_EXEC_MODE)}
    try:
        _abi.msf_set_option(_abi.OPT_SHORTCUT, mode)
        _abi.msf_set_option(_abi.OPT_OS_THRESHOLD, 50)  # both branches of the optimized schedule occur
        for ex in (0, 1):
            _abi.msf_set_option(_abi.OPT_EXEC_MODE, ex)
            g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
            mk, lb, tt = g.compute()
            st = g.stats()
            g.free()
            got = (mk.cpu().numpy(), lb.cpu().numpy(), float(tt.cpu()[0]))
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"], got=got)
            ref = as_rounds.as_msf(d["n"], d["src"], d["dst"], d["w"], d["wtype"], mode=SCHEDULES[mode],
                                   max_rounds=500)
            assert st.rounds == expected_rounds(ref, mode)
    finally:
        for o, v in old.items():
            _abi.msf_set_option(o, v)


@pytest.mark.parametrize("mode", [0, 1])
def test_partial_forest_after_each_round(mode):
    """With the round limit at k the call stops after k rounds: the edge mask
    equals the oracle's after k rounds of the same schedule."""
    import torch
    from oracle import as_rounds
    from paper_2110_04865_gb300 import _abi, api
    lib = _abi.load()
    d = synth.workload("grid16")
    full = as_rounds.as_msf(d["n"], d["src"], d["dst"], d["w"], 1, mode=SCHEDULES[mode], max_rounds=500)
    old = {o: _abi.msf_get_option(o) for o in (_abi.OPT_SHORTCUT, _abi.OPT_ROUND_LIMIT)}
    g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    try:
        _abi.msf_set_option(_abi.OPT_SHORTCUT, mode)
        for k in range(1, expected_rounds(full, mode)):
            _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, k)
            mk = torch.empty(len(d["src"]), dtype=torch.uint8, device=DEV)
            rc = lib.msf_compute(g.handle, mk.data_ptr(), None, None, None)
            assert rc == 4
            part = as_rounds.as_msf(d["n"], d["src"], d["dst"], d["w"], 1, mode=SCHEDULES[mode], stop_after=k)
            assert np.array_equal(mk.cpu().numpy(), part["mask"]), k
    finally:
        g.free()
        for o, v in old.items():
            _abi.msf_set_option(o, v)


@pytest.mark.parametrize("workload", ["rmat16p", "rmat20p"])
def test_permuted_rmat(workload):
    """R-MAT with permuted vertex ids (hubs spread over the id range and the
    builder's buckets): same oracle parity."""
    d = synth.workload(workload)
    assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"])


@pytest.mark.parametrize("workload", ["er4096", "rmat16", "grid64", "rmat20"])
def test_connected_components_workloads(workload):
    """Awerbuch-Shiloach connectivity (Sec. 2.4) on the GPU: the labels are
    the oracle's component labels and the round count is the step oracle's."""
    from oracle import as_cc
    from paper_2110_04865_gb300 import api
    d = synth.workload(workload)
    g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    lb = g.components().cpu().numpy()
    st = g.stats()
    g.free()
    _, olb, _ = oracle.kruskal(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
    assert np.array_equal(lb, olb)
    if d["n"] <= 300000:
        assert st.cc_rounds == as_cc.as_cc(d["n"], d["src"], d["dst"])["rounds"]


@pytest.mark.parametrize("seed", range(8))
def test_connected_components_random(seed):
    from oracle import as_cc
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(70 + seed)
    n = int(rng.integers(1, 4000))
    m = int(rng.integers(0, 3 * n))
    src, dst, w = rand_graph(rng, n, m, 0)
    g = api.Graph(n, to_dev(src), to_dev(dst), to_dev(w))
    lb = g.components().cpu().numpy()
    st = g.stats()
    g.free()
    ref = as_cc.as_cc(n, src, dst)
    assert np.array_equal(lb, ref["labels"])
    assert st.cc_rounds == ref["rounds"]


def _cc_partial_labels(g, n, k):
    """Labels after at most k connectivity rounds (round limit k) through the
    C ABI; returns (labels, rc, rounds)."""
    import torch
    from paper_2110_04865_gb300 import _abi
    lib = _abi.load()
    old = _abi.msf_get_option(_abi.OPT_ROUND_LIMIT)
    try:
        _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, k)
        lb = torch.empty(n, dtype=torch.int32, device=DEV)
        rc = lib.msf_connected_components(g.handle, lb.data_ptr(), None)
        return lb.cpu().numpy(), rc, int(_abi.msf_get_stats(g.handle).cc_rounds)
    finally:
        _abi.msf_set_option(_abi.OPT_ROUND_LIMIT, old)


@pytest.mark.parametrize("case", ["fixture", "random3", "random5", "rmat16"])
def test_connected_components_after_each_round(case):
    """Round by round (round limit k): the trees the GPU holds after k rounds
    are the step oracle's after k rounds (compared through their smallest
    vertex ids); the hand-worked fixture pins the oracle's trajectory."""
    from golden_io import connectivity_fixtures
    from oracle import as_cc
    from paper_2110_04865_gb300 import api
    if case == "fixture":
        fx = connectivity_fixtures()[0]
        n, src, dst = fx["n"], fx["src"], fx["dst"]
    elif case == "rmat16":
        d = synth.workload("rmat16")
        n, src, dst = d["n"], d["src"], d["dst"]
    else:
        rng = np.random.default_rng(70 + int(case[-1]))
        n = int(rng.integers(1, 4000))
        m = int(rng.integers(0, 3 * n))
        src, dst, _ = rand_graph(rng, n, m, 0)
    full = as_cc.as_cc(n, src, dst)
    w = np.ones(len(src), np.float32)
    g = api.Graph(n, to_dev(src), to_dev(dst), to_dev(w))
    try:
        for k in range(1, full["rounds"] + 1):
            lb, rc, rounds = _cc_partial_labels(g, n, k)
            assert rc == (0 if k == full["rounds"] else 4), k
            assert rounds == k
            part = as_cc.as_cc(n, src, dst, stop_after=k)
            assert np.array_equal(lb, part["labels"]), k
    finally:
        g.free()


def test_connected_components_repeat_deterministically():
    """The same graph twenty times: the same round count and labels every time
    (the random graph that exposed two stars hooking onto each other)."""
    from oracle import as_cc
    from paper_2110_04865_gb300 import api
    rng = np.random.default_rng(75)
    n = int(rng.integers(1, 4000))
    m = int(rng.integers(0, 3 * n))
    src, dst, w = rand_graph(rng, n, m, 0)
    ref = as_cc.as_cc(n, src, dst)
    g = api.Graph(n, to_dev(src), to_dev(dst), to_dev(w))
    try:
        for _ in range(20):
            lb = g.components().cpu().numpy()
            assert g.stats().cc_rounds == ref["rounds"]
            assert np.array_equal(lb, ref["labels"])
    finally:
        g.free()


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("workload", ["er4096", "rmat16", "grid16"])
def test_builders_agree(mode, workload):
    """The atomic-counter, radix and bucketed CSR builders give the same forest."""
    from paper_2110_04865_gb300 import _abi
    d = synth.workload(workload)
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, mode)
        assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


@pytest.mark.parametrize("n,m", [(1, 0), (2, 1), (5, 7), (16384, 1), (16385, 33333), (40000, 99999),
                                 (70000, 400001)])
def test_bucket_builder_edge_cases(n, m):
    """Bucketed builder: one or several buckets of 2^14 vertices, a partial
    last bucket, odd edge counts (the unpaired last edge of a block's chunk),
    self-loops and duplicate edges, buckets split into several work items."""
    from paper_2110_04865_gb300 import _abi
    rng = np.random.default_rng(n * 7 + m)
    s, d, w = rand_graph(rng, n, m, 0)
    if m > 6:
        s[:3] = d[:3]  # self-loops
        s[-2:], d[-2:], w[-2:] = s[3:5], d[3:5], w[3:5]  # duplicate edges, equal weights
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, 3)
        assert_parity(n, s, d, w, 0)
        s2, d2, w2 = rand_graph(rng, n, m, 1, levels=7)
        assert_parity(n, s2, d2, w2, 1)
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


def test_bucket_builder_wide_buckets():
    """Bucketed builder on graphs with more than 2^22 vertices: buckets wider
    than 4096 rows, split again into sub-buckets of 512 rows (a hub bucket
    spread over many chunks of the second partition)."""
    from paper_2110_04865_gb300 import _abi
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, 3)
        rng = np.random.default_rng(11)
        for n, m in ((1 << 23, 3000017), (9000000, 1 << 22)):
            s, d, w = rand_graph(rng, n, m, 0)
            s[: m // 4] = rng.integers(0, 64, m // 4)  # a few high-degree rows
            assert_parity(n, s, d, w, 0)
        dd = synth.workload("grid128")
        assert_parity(dd["n"], dd["src"], dd["dst"], dd["w"], dd["wtype"])
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


def test_bucket_builder_multi_bucket_workloads():
    """Bucketed builder on R-MAT 20 (512 buckets of 2048 rows, the first ones
    split into hundreds of work items; one-word records), on a graph of 3
    million vertices (4096-row buckets, two-word records) and on a batch of
    graphs (global ids)."""
    from paper_2110_04865_gb300 import _abi, api
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, 3)
        d = synth.workload("rmat20")
        assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
        rng = np.random.default_rng(23)
        n3, m3 = 3_000_000, 1 << 21
        s3, d3, w3 = rand_graph(rng, n3, m3, 1)
        d3[: m3 // 8] = rng.integers(0, 16, m3 // 8)  # a few high-degree rows
        assert_parity(n3, s3, d3, w3, 1)
        b = synth.batch(64, seed=77)
        voff, eoff, s, dd, w = b[:5]
        mk, lb, tt = api.compute_batched(voff, eoff, to_dev(s), to_dev(dd), to_dev(w))
        _abi.msf_set_option(_abi.OPT_BUILD, 1)
        mk1, lb1, tt1 = api.compute_batched(voff, eoff, to_dev(s), to_dev(dd), to_dev(w))
        assert np.array_equal(mk.cpu().numpy(), mk1.cpu().numpy())
        assert np.array_equal(lb.cpu().numpy(), lb1.cpu().numpy())
        assert np.array_equal(tt.cpu().numpy(), tt1.cpu().numpy())
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


def test_automatic_builder_choice():
    """From 2^20 edges the automatic choice takes the bucketed builder for
    scattered edge lists (R-MAT 20, its permuted form) and the per-vertex
    atomic one for edge lists with locality (the 128^3 lattice listed vertex
    by vertex, a batch listed graph by graph); the forests are the oracle's."""
    from paper_2110_04865_gb300 import _abi, api
    old = _abi.msf_get_option(_abi.OPT_BUILD)
    try:
        _abi.msf_set_option(_abi.OPT_BUILD, 0)
        for wl, want in (("rmat20", 3), ("rmat20p", 3), ("grid128", 1)):
            d = synth.workload(wl)
            g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
            assert g.stats().builder == want, wl
            got = g.compute()
            g.free()
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"],
                          got=(got[0].cpu().numpy(), got[1].cpu().numpy(), float(got[2].cpu()[0])))
        voff, eoff, s_, d_, w_ = synth.batch(256, seed=5)[:5]
        assert eoff[-1] >= 1 << 20
        # the batch as one graph with global ids
        gs = (s_.astype(np.int64) + np.repeat(voff[:-1], np.diff(eoff))).astype(np.int32)
        gd = (d_.astype(np.int64) + np.repeat(voff[:-1], np.diff(eoff))).astype(np.int32)
        g = api.Graph(int(voff[-1]), to_dev(gs), to_dev(gd), to_dev(w_))
        assert g.stats().builder == 1
        g.free()
    finally:
        _abi.msf_set_option(_abi.OPT_BUILD, old)


@pytest.mark.parametrize("sweep", [1, 2])
@pytest.mark.parametrize("spl", [4, 8, 16])
@pytest.mark.parametrize("workload", ["er4096", "rmat16", "grid16", "grid64"])
def test_pipelined_sweep_gives_the_same_results(sweep, spl, workload):
    """The pipelined sweeps (1: shared-memory stages filled by bulk copies two
    tiles ahead; 2: register tiles two ahead with gathers one ahead) give the
    same forest as the oracle (with compactions on grid64) and the same
    min-edge vector as the register-tile sweep, for the identity and for a
    random parent vector."""
    import torch
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload(workload)
    old = {o: _abi.msf_get_option(o) for o in (_abi.OPT_SWEEP, _abi.OPT_SLOTS_PER_LANE)}
    try:
        _abi.msf_set_option(_abi.OPT_SLOTS_PER_LANE, spl)
        _abi.msf_set_option(_abi.OPT_SWEEP, sweep)
        assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
        g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
        rng = np.random.default_rng(spl)
        for par in (np.arange(d["n"], dtype=np.int32), rng.integers(0, max(d["n"] // 7, 1), d["n"]).astype(np.int32)):
            pt = torch.from_numpy(par).to(DEV)
            _abi.msf_set_option(_abi.OPT_SWEEP, sweep)
            r1 = g.min_edge(pt).clone()
            _abi.msf_set_option(_abi.OPT_SWEEP, 0)
            r0 = g.min_edge(pt)
            assert torch.equal(r0, r1)
        g.free()
    finally:
        for o, v in old.items():
            _abi.msf_set_option(o, v)


@pytest.mark.parametrize("workload", ["er4096", "rmat16", "rmat20", "grid64"])
@pytest.mark.parametrize("tau", [0.0, 0.9])
def test_relabelled_columns_give_the_same_results(workload, tau):
    """With the second round's sweep writing the columns as their roots
    (MSF_OPT_RELABEL, the default) and without it: the oracle's forest, the
    same rounds, and twice on one graph (the relabelled copy never replaces
    the graph's own columns); with compactions too (tau 0.9)."""
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload(workload)
    old = {o: _abi.msf_get_option(o) for o in (_abi.OPT_RELABEL, _abi.OPT_COMPACT_TAU)}
    g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    try:
        _abi.msf_set_option(_abi.OPT_COMPACT_TAU, tau)
        rounds = {}
        for rel in (1, 0, 1):
            _abi.msf_set_option(_abi.OPT_RELABEL, rel)
            mk, lb, tt = g.compute()
            got = (mk.cpu().numpy(), lb.cpu().numpy(), float(tt.cpu()[0]))
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"], got=got)
            rounds.setdefault(rel, set()).add(int(g.stats().rounds))
        assert len(rounds[1]) == 1 and rounds[1] == rounds[0]
    finally:
        g.free()
        for o, v in old.items():
            _abi.msf_set_option(o, v)


@pytest.mark.parametrize("workload", ["rmat12", "grid16", "er4096"])
def test_pairwise_kernel_gives_the_same_forest(workload):
    """The pairwise formulation of Sec. 4.1 (p_j materialised next to every
    slot, then reduced) gives the same forest and the same min-edge result."""
    import torch
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload(workload)
    old = _abi.msf_get_option(_abi.OPT_KERNEL)
    try:
        _abi.msf_set_option(_abi.OPT_KERNEL, 1)
        assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
        g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
        p = torch.arange(d["n"], dtype=torch.int32, device=DEV)
        r1 = g.min_edge(p).clone()
        _abi.msf_set_option(_abi.OPT_KERNEL, 0)
        r0 = g.min_edge(p)
        g.free()
        assert torch.equal(r0, r1)
    finally:
        _abi.msf_set_option(_abi.OPT_KERNEL, old)


@pytest.mark.parametrize("workload", ["rmat16", "grid64"])
def test_early_stop_off_runs_the_confirming_round(workload):
    from oracle import as_rounds
    from paper_2110_04865_gb300 import _abi, api
    d = synth.workload(workload)
    ref = as_rounds.as_msf(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
    rounds = {}
    old = _abi.msf_get_option(_abi.OPT_EARLY_STOP)
    try:
        for es in (0, 1):
            _abi.msf_set_option(_abi.OPT_EARLY_STOP, es)
            g = api.Graph(d["n"], to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
            got = tuple(x.cpu().numpy() for x in g.compute())
            rounds[es] = g.stats().rounds
            g.free()
            assert_parity(d["n"], d["src"], d["dst"], d["w"], d["wtype"], got=(got[0], got[1], float(got[2][0])))
    finally:
        _abi.msf_set_option(_abi.OPT_EARLY_STOP, old)
    assert rounds[0] == ref["rounds"]
    assert rounds[1] == expected_rounds(ref, 0)
