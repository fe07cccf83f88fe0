"""msf_forest_weight_noalloc: the forest weight computed with no device
allocation, for callers that cannot allocate device memory at call time
(another allocator owns the memory budget, the host application forbids
cudaMalloc/cudaFree, or the caller cannot afford their implicit device
synchronisation).  Its scratch is a fixed array in the library's device image.

Checked through the C ABI against the totals msf_compute_batched and
msf_compute return for the same forests, exactly (the tests' tolerance for
totals), on two calls in a row: the shared scratch must be cleared by each
call.  This file is collected last so that a failure here stops a -x run only
after every other test has run."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_04865_gb300 import _abi, build_lib
    build_lib.build()
    return torch, _abi, _abi.load()


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda:0")


def test_noalloc_weight_matches_batched_totals(env):
    torch, _abi, lib = env
    from paper_2110_04865_gb300 import api
    G = 300
    voff, eoff, s, d, w, _ = synth.batch(G, nmax=4096, seed=31)
    wd = _dev(torch, w)
    mask, _, totals = api.compute_batched(voff, eoff, _dev(torch, s), _dev(torch, d), wd)
    eo = np.ascontiguousarray(eoff, dtype=np.int64)
    stream = int(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((G,), float("nan"), dtype=torch.float64, device="cuda:0")
        rc = lib.msf_forest_weight_noalloc(G, int(eo[-1]), eo.ctypes.data, mask.data_ptr(), wd.data_ptr(),
                                           0, out.data_ptr(), stream or None)
        assert rc == 0, _abi.msf_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, totals)


def test_noalloc_weight_matches_single_graph_u32(env):
    torch, _abi, lib = env
    from paper_2110_04865_gb300 import api
    dd = synth.workload("grid16")
    wd = _dev(torch, dd["w"])
    mask, _, total = api.compute(dd["n"], _dev(torch, dd["src"]), _dev(torch, dd["dst"]), wd)
    stream = int(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        _abi.msf_forest_weight_noalloc(1, len(dd["src"]), 0, mask.data_ptr(), wd.data_ptr(), 1, out.data_ptr(),
                                       stream)
        torch.cuda.synchronize()
        assert torch.equal(out, total)


def test_noalloc_weight_rejects_beyond_maximum_and_host_buffers(env):
    torch, _abi, lib = env
    eo = np.zeros(1026, np.int64)
    out = torch.zeros(1025, dtype=torch.float64, device="cuda:0")
    rc = lib.msf_forest_weight_noalloc(1025, 0, eo.ctypes.data, None, None, 0, out.data_ptr(), None)
    assert rc == 6 and b"1024" in lib.msf_last_error()
    hm = np.ones(4, np.uint8)
    hw = np.ones(4, np.float32)
    rc = lib.msf_forest_weight_noalloc(1, 4, None, hm.ctypes.data, hw.ctypes.data, 0, out.data_ptr(), None)
    assert rc == 1 and b"device memory" in lib.msf_last_error()


def test_noalloc_weight_nan_weight_gives_nan(env):
    """A selected NaN weight makes its graph's total NaN (the other graphs'
    totals are unaffected), on two calls in a row."""
    torch, _abi, lib = env
    w = torch.tensor([1.0, float("nan"), 2.0, 0.5], dtype=torch.float32, device="cuda:0")
    mask = torch.tensor([1, 1, 1, 1], dtype=torch.uint8, device="cuda:0")
    eo = np.array([0, 2, 4], np.int64)
    stream = int(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
        rc = lib.msf_forest_weight_noalloc(2, 4, eo.ctypes.data, mask.data_ptr(), w.data_ptr(), 0,
                                           out.data_ptr(), stream or None)
        assert rc == 0, _abi.msf_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.isnan(o[0]) and o[1] == 2.5
