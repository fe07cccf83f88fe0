"""bench.py's reference arm (the CPU oracle) on a small workload, no GPU:
the JSON line carries the keys the measurement contract asks for."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra=None, *args):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "er4096", "--steps", "2", "--warmup", "1", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] >= 3  # at least three warm-up steps, whatever is asked
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("Erdos-Renyi")


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_clock_summary_reads_nvidia_smi_samples(tmp_path):
    """The clocks record of the bench line from nvidia-smi's CSV (index, SM
    clock, max SM clock, power, active-reasons mask, then hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""
    sys.path.insert(0, ROOT)
    import bench
    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1995, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n"
                 "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not p.exists()  # the sample file is removed
    p.write_text("0, 1410, 2070, 500, 0x8, Active, Not Active, Active, Not Active\n")
    cs.path = str(p)
    s = cs.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1410.0
    cs.path = str(tmp_path / "missing.csv")
    assert cs.summary()["reasons"] == ["unsampled"]
