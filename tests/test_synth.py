"""The seeded generators: determinism, sizes and value ranges (no GPU)."""
import numpy as np

import synth


def test_counter_based_and_deterministic():
    a = synth.er(1000, 5000, seed=5)
    b = synth.er(1000, 5000, seed=5)
    c = synth.er(1000, 2000, seed=5)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        assert np.array_equal(x[:2000], z)          # prefix of the same counters
    assert not np.array_equal(a[0], synth.er(1000, 5000, seed=6)[0])


def test_weight_encodings():
    _, _, w = synth.er(100, 20000, wtype=0)
    k = (w.astype(np.float64) * 2 ** 24 - 1) / 2
    assert np.all(k == np.floor(k)) and w.min() > 0 and w.max() < 1
    _, _, u = synth.er(100, 20000, wtype=1)
    assert u.dtype == np.uint32 and u.min() >= 1 and u.max() <= 1000


def test_rmat_and_grid_shapes():
    s, d, w = synth.rmat(10, 16)
    assert len(s) == 16 << 10 and s.max() < 1024 and d.max() < 1024
    # skew: vertex 0 (all-zero bits) is the most likely endpoint
    deg = np.bincount(np.concatenate([s, d]), minlength=1024)
    assert deg.argmax() == 0
    s, d, w = synth.grid3d(4, 3, 2)
    assert len(s) == 3 * 3 * 2 + 4 * 2 * 2 + 4 * 3 * 1 == synth.grid3d_count(4, 3, 2)
    assert np.all(np.isin(d - s, [1, 4, 12]))
    assert synth.grid3d_count(256, 256, 256) == 3 * 256 * 256 * 255


def test_rgg_and_batch():
    s, d, w = synth.rgg(5000, 8.0)
    assert np.all(s < d) and abs(2 * len(s) / 5000 - 8.0) < 1.0
    voff, eoff, s, d, w, kind = synth.batch(64, nmin=64, nmax=4096)
    nv = np.diff(voff)
    assert nv.min() >= 64 and nv.max() <= 4096 and len(s) == eoff[-1]
    for g in range(64):
        a, b = eoff[g], eoff[g + 1]
        assert s[a:b].max(initial=0) < nv[g] and d[a:b].max(initial=0) < nv[g]


def test_permuted_rmat_is_a_relabelling():
    """rmat<scale>p is the same multigraph under a bijection of the vertex ids."""
    p = synth.permutation(12)
    assert np.array_equal(np.sort(p), np.arange(1 << 12))
    a, b = synth.workload("rmat12"), synth.workload("rmat12p")
    assert np.array_equal(b["src"], p[a["src"]]) and np.array_equal(b["dst"], p[a["dst"]])
    assert np.array_equal(a["w"], b["w"]) and a["n"] == b["n"]
    assert p[0] != 0  # the largest hub moves away from id 0
