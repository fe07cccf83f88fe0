"""Host logic of the autotuner (no GPU): which measured candidate it keeps."""
from __future__ import annotations

import pytest

pytest.importorskip("torch")

from paper_2110_04865_gb300 import autotune  # noqa: E402


def test_shape_is_the_fastest_unless_a_near_tie_sweeps_faster():
    # (ms, sweep_ms, spl, prefetch, blocks_per_sm, sweep)
    table = [(10.0, 2.0, 4, 0, 4, 0), (9.0, 3.0, 8, 0, 8, 0), (12.0, 1.0, 16, 0, 2, 0)]
    assert autotune.pick_shape(table)[2:] == (8, 0, 8, 0)
    # within 1 % of the fastest round loop, the faster full sweep wins
    table = [(9.05, 2.5, 4, 1, 8, 0), (9.0, 3.0, 8, 0, 8, 0), (9.2, 1.0, 16, 0, 2, 0)]
    assert autotune.pick_shape(table)[2:] == (4, 1, 8, 0)


def test_first_candidate_wins_a_near_tie():
    # compaction thresholds in candidate order: the default (first) within 1 %
    assert autotune.pick_first([(10.05, 0.5), (10.0, 0.25), (11.0, 0.0)]) == (10.05, 0.5)
    assert autotune.pick_first([(10.5, 0.5), (10.0, 0.25), (10.09, 0.0)]) == (10.0, 0.25)
    # batched shapes (ms, spl, prefetch, blocks_per_sm, sweep)
    rows = [(25.0, 4, 0, 2, 0), (24.1, 8, 0, 4, 0), (24.0, 8, 1, 4, 0)]
    assert autotune.pick_first(rows) == (24.1, 8, 0, 4, 0)


def test_every_candidate_is_a_valid_shape():
    seen = set()
    for spl, pf, bps, sw in autotune.CANDIDATES:
        assert spl in (4, 8, 16) and pf in (0, 1) and 1 <= bps <= 8 and sw in (0, 1, 2)
        assert (spl, pf, bps, sw) not in seen
        seen.add((spl, pf, bps, sw))
    assert autotune.TAU_CANDIDATES[0] == 0.5  # the library's default first
