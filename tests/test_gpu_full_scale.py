"""R-MAT scale 26 (2^26 vertices, 2^30 edges, ~2.15e9 CSR slots): GPU forest
vs the full CPU oracle, bit for bit, in the launch configuration the benchmark
times (automatic builder, default sweep shape).  Needs ~80 GB of device
memory, ~40 GB of host memory and about a minute and a half of
single-threaded Kruskal."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_rmat26_full_parity():
    import torch
    from paper_2110_04865_gb300 import api, build_lib
    build_lib.build()
    t0 = time.time()
    d = synth.workload("rmat26")
    n, s, dd, w = d["n"], d["src"], d["dst"], d["w"]
    t_gen = time.time() - t0
    g = api.Graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(dd).cuda(), torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    t1 = time.time()
    mk, lb, tt = g.compute()
    torch.cuda.synchronize()
    t_gpu = time.time() - t1
    st = g.stats()
    g.free()
    mk = mk.cpu().numpy()
    lb = lb.cpu().numpy()
    tot = float(tt.cpu()[0])
    torch.cuda.empty_cache()
    t2 = time.time()
    omk, olb, otot = oracle.kruskal(n, s, dd, w, 0)
    t_cpu = time.time() - t2
    print(f"\nrmat26: gen {t_gen:.1f}s gpu compute {t_gpu * 1e3:.1f} ms oracle {t_cpu:.1f}s "
          f"rounds {st.rounds} compactions {st.compactions} forest {st.forest_edges} nnz {st.nnz}")
    assert np.array_equal(mk, omk)
    assert np.array_equal(lb, olb)
    assert tot == otot
