"""The partitioned round loop through the library (GPU): msf_min_edge_part
sweeps one part of a 1-D partition of the CSR's slots (Sec. 4.1's
distribution of A, one part per process), a MIN reduction joins the partial
projections, and msf_apply_round hooks, breaks ties and shortcuts on
replicated parents.  Checked against msf_min_edge and against the oracle's
forest: in one process over several parts, and with two gloo ranks that
share cuda:0 and join their keys over gloo on host copies (no peer memory;
no kernel of one rank waits on the other)."""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import DEV, to_dev

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_04865_gb300 import build_lib
    build_lib.build()


def _graph(name):
    if name == "er":
        d = synth.workload("er4096")
    elif name == "ties":
        rng = np.random.default_rng(17)
        n, m = 5000, 40000
        d = dict(n=n, src=rng.integers(0, n, m).astype(np.int32), dst=rng.integers(0, n, m).astype(np.int32),
                 w=rng.choice(np.linspace(0.1, 1, 4), m).astype(np.float32), wtype=0)
    else:
        d = synth.workload(name)
    return d


@pytest.mark.parametrize("nparts", [1, 2, 3, 7, 64])
def test_parts_join_to_the_full_projection(nparts):
    """min over the parts of msf_min_edge_part == msf_min_edge, for the
    identity parents and for the star forest after one round."""
    import torch
    from oracle import as_rounds
    from paper_2110_04865_gb300 import _abi, api
    d = _graph("rmat16")
    n = d["n"]
    g = api.Graph(n, to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    try:
        one = as_rounds.as_msf(n, d["src"], d["dst"], d["w"], 0, stop_after=1)["parent"]
        for par in (np.arange(n, dtype=np.int32), one.astype(np.int32)):
            p = to_dev(par)
            full = torch.empty(n, dtype=torch.int64, device=DEV)
            _abi.msf_min_edge(g.handle, p.data_ptr(), full.data_ptr())
            joined = None
            for k in range(nparts):
                r = torch.empty(n, dtype=torch.int64, device=DEV)
                _abi.msf_min_edge_part(g.handle, p.data_ptr(), k, nparts, r.data_ptr())
                ru = r.cpu().numpy().view(np.uint64)
                joined = ru if joined is None else np.minimum(joined, ru)
            assert np.array_equal(joined, full.cpu().numpy().view(np.uint64))
    finally:
        g.free()


@pytest.mark.parametrize("name", ["er", "ties", "rmat16", "grid16"])
@pytest.mark.parametrize("nparts", [2, 5])
def test_partitioned_loop_in_one_process(name, nparts):
    """All parts swept in one process, joined by an elementwise minimum, then
    applied: the oracle's forest and labels."""
    import torch
    from paper_2110_04865_gb300 import _abi, api
    d = _graph(name)
    n, m = d["n"], len(d["src"])
    g = api.Graph(n, to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))
    try:
        parent = torch.arange(n, dtype=torch.int32, device=DEV)
        mask = torch.zeros(m, dtype=torch.uint8, device=DEV)
        labels = torch.empty(n, dtype=torch.int32, device=DEV)
        r = torch.empty(n, dtype=torch.int64, device=DEV)
        for rounds in range(1, 65):
            joined = None
            for k in range(nparts):
                _abi.msf_min_edge_part(g.handle, parent.data_ptr(), k, nparts, r.data_ptr())
                ru = r.cpu().numpy().view(np.uint64)
                joined = ru.copy() if joined is None else np.minimum(joined, ru)
            r.copy_(torch.from_numpy(joined.view(np.int64)))
            hooks = _abi.msf_apply_round(g.handle, r.data_ptr(), parent.data_ptr(), mask.data_ptr(),
                                         labels.data_ptr())
            assert np.all(r.cpu().numpy().view(np.uint64) == np.uint64(0xFFFFFFFFFFFFFFFF))
            if hooks == 0:
                break
        omk, olb, _ = oracle.kruskal(n, d["src"], d["dst"], d["w"], d["wtype"])
        assert np.array_equal(mask.cpu().numpy(), omk)
        assert np.array_equal(labels.cpu().numpy(), olb)
    finally:
        g.free()


def test_apply_round_rejects_a_foreign_projection():
    """A key whose edge does not leave the root's star is reported
    (MSF_ERR_CHECK), not applied."""
    import torch
    from paper_2110_04865_gb300 import _abi, api
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 3], np.int32)
    w = np.array([1.0, 2.0, 3.0], np.float32)
    g = api.Graph(4, to_dev(src), to_dev(dst), to_dev(w))
    try:
        parent = torch.arange(4, dtype=torch.int32, device=DEV)
        mask = torch.zeros(3, dtype=torch.uint8, device=DEV)
        # vertex 3 claims edge 0 = (0, 1), which does not touch it
        r = torch.tensor([-1, -1, -1, 0], dtype=torch.int64, device=DEV)
        with pytest.raises(_abi.MsfError) as ei:
            _abi.msf_apply_round(g.handle, r.data_ptr(), parent.data_ptr(), mask.data_ptr(), 0)
        assert ei.value.code == 7
    finally:
        g.free()


def _rank(rank, ws, port, name, queue):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        from paper_2110_04865_gb300 import api
        from paper_2110_04865_gb300.shard import solve_partitioned
        d = _graph(name)
        n, m = d["n"], len(d["src"])
        g = api.Graph(n, to_dev(d["src"]), to_dev(d["dst"]), to_dev(d["w"]))

        def allreduce_min(x):
            t = torch.from_numpy(np.ascontiguousarray(x))
            dist.all_reduce(t, op=dist.ReduceOp.MIN)
            return t.numpy()

        mask, labels, rounds = solve_partitioned(g.handle, n, m, rank, ws, allreduce_min, torch.device(DEV))
        torch.cuda.synchronize()
        queue.put((rank, mask.cpu().numpy(), labels.cpu().numpy(), rounds))
        g.free()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["ties", "rmat16"])
def test_two_gloo_ranks_on_one_gpu(name):
    mp = pytest.importorskip("torch.multiprocessing")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, queue)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted([queue.get(timeout=300) for _ in range(2)], key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    d = _graph(name)
    omk, olb, _ = oracle.kruskal(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
    for _, mk, lb, rounds in got:
        assert np.array_equal(mk, omk) and np.array_equal(lb, olb)
    assert got[0][3] == got[1][3]
