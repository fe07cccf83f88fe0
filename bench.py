"""Benchmark: undirected edges/s to the full minimum spanning forest.

One step = one pass of the whole hot path over one synthetic graph already
resident in HBM: msf_build_csr (CSR build and symmetrisation) + msf_compute
(the device round loop: min-edge sweeps, compaction, hooking, tie breaking,
complete shortcutting, labels, exact total) + msf_free.  Default workload:
R-MAT scale 26 (n = 2^26, 16 * 2^26 draws, a,b,c,d = .57,.19,.19,.05), float32
weights uniform in (0,1), the largest single-GPU configuration.  L2 is
flushed (a 256 MiB write) before every timed step (the inputs are also far
larger than L2); each step is timed with CUDA events on the current stream.

Also reported on the same JSON line:
  e2e           the same metric through the C ABI with pinned HOST buffers
                (host->device copies of the COO and device->host copies of
                mask, labels and total inside the timed region);
  roofline      the min-edge sweep (one msf_min_edge launch over every slot,
                timed with CUDA events) against the measured HBM copy peak;
  cpu_baseline  the CPU oracle (single-threaded Kruskal) on a bounded sample
                of the same graph (the prefix of its edge list beyond 2^26
                edges), with the host's core count and CPU model;
  cpu_baseline_all_cores  the same with the keys sorted on every host core;
  batched       one msf_compute_batched call on 4096 uneven graphs vs a loop
                of per-graph build + compute + free calls on the same GPU;
  pairwise_vs_multilinear  the Sec. 4.1 ablation on R-MAT 17, edge factor 8:
                round loop and full sweep, fused kernel vs two-pass form.
With --impl reference the CPU oracle is timed as the reference arm.
Under torchrun (N > 1) every rank solves its own replica of the workload
(the forest of one graph is not sharded); value = all ranks' edges / max time.
The batched leg shards its graphs: every rank solves a contiguous range of
them (balanced by edges, no exchange); its times are the slowest rank's.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "undirected edges/s to full MSF; min-edge kernel % HBM peak; batched vs looped"


def workload_desc(name: str) -> str:
    if name.startswith("rmat") and name.endswith("p"):
        return workload_desc(name[:-1]) + ", vertex ids permuted"
    if name.startswith("rmat"):
        body = name[4:]
        s, ef = (int(body.split("e")[0]), int(body.split("e")[1])) if "e" in body else (int(body), 16)
        return f"R-MAT scale {s} (n=2^{s}, edge factor {ef}, a=.57 b=.19 c=.19 d=.05), f32 weights in (0,1)"
    if name == "er4096":
        return "Erdos-Renyi n=4096 m=32768, f32 weights in (0,1)"
    if name == "er20":
        return "uniform random n=2^20 m=16*2^20, f32 weights in (0,1)"
    if name.startswith("grid"):
        k = int(name[4:])
        return f"3-D 7-point grid {k}^3, u32 weights in [1,1000]"
    return name


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# The CPU oracle is timed on a bounded sample of the workload: graphs with at
# most this many edges whole, larger ones by the prefix of their edge list
# (every edge of the synthetic generators is an independent draw, so the
# prefix is a graph of the same kind on the same vertex set).
CPU_SAMPLE_EDGES = 1 << 26


def host_info() -> dict:
    """The host the CPU baselines ran on: logical CPU count and CPU model."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


def cpu_sample(d: dict, name: str):
    """(sample dict, description) of the graph the CPU oracle is timed on."""
    m = len(d["src"])
    if m <= CPU_SAMPLE_EDGES:
        return d, f"full {name} graph ({m} edges)"
    k = CPU_SAMPLE_EDGES
    sd = dict(n=d["n"], src=d["src"][:k], dst=d["dst"][:k], w=d["w"][:k], wtype=d["wtype"])
    return sd, (f"the first {k} of the {m} edges of {name} (n = {d['n']}): the prefix of "
                "the same independent edge draws, i.e. the same generator with 1/"
                f"{m // k} of the edges")


def time_oracle(d, reps: int = 1, threads: int = 0):
    """Best wall time of the CPU oracle on d: the single-threaded Kruskal
    (threads = 0), or its variant that sorts the keys on `threads` threads
    before the same sequential union-find scan."""
    import oracle
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        if threads:
            oracle.kruskal_mt(d["n"], d["src"], d["dst"], d["w"], d["wtype"], threads)
        else:
            oracle.kruskal(d["n"], d["src"], d["dst"], d["w"], d["wtype"])
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best


def run_reference(args):
    """Reference arm: the CPU oracle (Kruskal + union-find), single thread,
    one bounded sample of the workload per step."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    d = synth.workload(args.workload)
    n, m_full = d["n"], len(d["src"])
    sd, sample = cpu_sample(d, args.workload)
    m = len(sd["src"])
    for _ in range(args.warmup):
        time_oracle(sd)
    times = [time_oracle(sd) for _ in range(args.steps)]
    tot = sum(times)
    value = m * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 keys (f32 weight order + edge id)",
        "data": "synthetic", "config": {"workload": workload_desc(args.workload), "n": n, "m": m_full},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": sample + ", once per step", "host": host_info()},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# the sources of the min-edge sweep: a traffic capture stays valid while these are unchanged
SWEEP_SOURCES = ("minedge.cu", "internal.cuh")


def env_shape():
    """The sweep shape MSF_SPL / MSF_PREFETCH / MSF_BPS / MSF_SWEEP select (the
    library's defaults where unset)."""
    return {"spl": int(os.environ.get("MSF_SPL", "4")), "prefetch": int(os.environ.get("MSF_PREFETCH", "0")),
            "blocks_per_sm": int(os.environ.get("MSF_BPS", "4")), "sweep": int(os.environ.get("MSF_SWEEP", "0"))}


def ingest_traffic(args):
    """profiles/min_edge_traffic.json from the ncu CSV of
    `bench.py --profile-min-edge --workload W` run with the sweep shape in
    MSF_SPL / MSF_PREFETCH / MSF_BPS / MSF_SWEEP (the shape the autotuner
    picks on W): the mean DRAM bytes (read + write) per captured k_sweep
    launch, each after an L2 flush.  Entries for other shapes of the same
    workload and sources are kept."""
    import csv

    from paper_2110_04865_gb300 import build_lib
    per = {}
    with open(args.ingest_traffic) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        # the sweep proper, not its relabelling instantiation (launched beside it,
        # it returns at once outside the second round of a round loop)
        if "k_sweep" not in r["Kernel Name"] or ", 1>(" in r["Kernel Name"]:
            continue
        unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(r.get("Metric Unit", "byte"), None)
        if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum") and unit:
            key = int(r["ID"])
            per[key] = per.get(key, 0.0) + float(r["Metric Value"].replace(",", "")) * unit
    if not per:
        raise SystemExit("no k_sweep DRAM counters in the capture")
    shape = env_shape()
    src_hash = build_lib.source_hash(SWEEP_SOURCES)
    path = os.path.join(ROOT, "profiles", "min_edge_traffic.json")
    caps = []
    try:
        old = json.load(open(path))
        if old.get("workload") == args.workload and old.get("source_hash") == src_hash:
            caps = [c for c in old.get("captures", []) if c.get("config") != shape]
    except (OSError, ValueError):
        pass
    caps.append({"config": shape, "dram_bytes_per_launch": int(sum(per.values()) / len(per)),
                 "launches": len(per)})
    env = " ".join(f"MSF_{k}={v}" for k, v in (("SPL", shape["spl"]), ("PREFETCH", shape["prefetch"]),
                                                ("BPS", shape["blocks_per_sm"]), ("SWEEP", shape["sweep"])))
    out = {"workload": args.workload, "source_hash": src_hash, "sources": list(SWEEP_SOURCES),
           "command": f"{env} ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                      f"--clock-control none -k regex:k_sweep -s 1 -c 4 --csv python bench.py --profile-min-edge "
                      f"--workload {args.workload} --no-autotune  (each msf_min_edge call launches the sweep and "
                      f"its relabelling instantiation, which returns at once outside a round loop's second "
                      f"round and is left out: the 4 captured launches hold 2 sweeps)",
           "captures": caps}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path} ({shape}: {caps[-1]['dram_bytes_per_launch']} bytes per launch)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-pairwise", action="store_true",
                    help="skip the multilinear vs pairwise ablation (R-MAT 17, edge factor 8)")
    ap.add_argument("--profile-min-edge", action="store_true",
                    help="only build the graph and run the min-edge sweep 4 times (for ncu)")
    ap.add_argument("--ingest-traffic", metavar="CSV",
                    help="read an ncu CSV of a --profile-min-edge capture (dram__bytes_read.sum, "
                         "dram__bytes_write.sum of k_sweep, the shape in MSF_SPL/MSF_PREFETCH/MSF_BPS/"
                         "MSF_SWEEP) and write profiles/min_edge_traffic.json")
    ap.add_argument("--profile-build", action="store_true",
                    help="only build (and free) the CSR 3 times (for ncu)")
    ap.add_argument("--profile-step", action="store_true",
                    help="only run the step (build + compute + free) twice, untimed (for an ncu launch list; "
                         "with --exec host every kernel of the round loop is a separate launch)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="only run msf_compute_batched on the 4096-graph batch 3 times (for ncu)")
    ap.add_argument("--exec", default="graph", choices=["graph", "host"],
                    help="round loop as a CUDA graph (default) or host-driven (kernels listed one by one under ncu)")
    ap.add_argument("--no-relabel", action="store_true",
                    help="leave the later rounds' sweeps on the original column array (MSF_OPT_RELABEL 0)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default sweep shape and compaction threshold (or the ones "
                         "MSF_SPL/MSF_PREFETCH/MSF_BPS/MSF_SWEEP/MSF_TAU give)")
    ap.add_argument("--build", default="auto", choices=["auto", "atomic", "radix", "bucket"])
    ap.add_argument("--kernel", default="multilinear", choices=["multilinear", "pairwise"],
                    help="min-edge formulation (pairwise = the two-pass ablation of Sec. 4.1)")
    ap.add_argument("--shortcut", default="csp", choices=["csp", "original", "full", "optimized"])
    ap.add_argument("--components", action="store_true",
                    help="time msf_connected_components on the workload instead (one JSON line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.ingest_traffic:
        ingest_traffic(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    import synth
    from paper_2110_04865_gb300 import _abi, build_lib

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build_lib.build()
    lib = _abi.load()
    if args.exec == "host":
        _abi.msf_set_option(_abi.OPT_EXEC_MODE, 1)
    _abi.msf_set_option(_abi.OPT_BUILD, {"auto": 0, "atomic": 1, "radix": 2, "bucket": 3}[args.build])
    _abi.msf_set_option(_abi.OPT_KERNEL, 1 if args.kernel == "pairwise" else 0)
    _abi.msf_set_option(_abi.OPT_SHORTCUT, ["csp", "original", "full", "optimized"].index(args.shortcut))
    if args.no_relabel:
        _abi.msf_set_option(_abi.OPT_RELABEL, 0)

    d = synth.workload(args.workload)
    n, m, wtype = d["n"], len(d["src"]), d["wtype"]
    wnp = d["w"].view(np.int32) if wtype == 1 else d["w"]
    src = torch.from_numpy(d["src"]).to(dev)
    dst = torch.from_numpy(d["dst"]).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(wnp)).to(dev)
    mask = torch.empty(m, dtype=torch.uint8, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    total = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = int(stream.cuda_stream)

    if args.components:
        from paper_2110_04865_gb300 import api
        g = api.Graph(n, src, dst, w)
        for _ in range(args.warmup):
            g.components()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.components()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        st = g.stats()
        g.free()
        t = statistics.median(ts)
        print(json.dumps({"metric": "connected components: undirected edges/s (Sec. 2.4, CSR resident)",
                          "value": m / (t / 1e3), "unit": "edges/s", "ms": t, "rounds": int(st.cc_rounds),
                          "config": {"workload": workload_desc(args.workload), "n": n, "m": m}}), flush=True)
        return

    if args.profile_build:
        _abi.msf_set_option(_abi.OPT_BUILD, {"auto": 0, "atomic": 1, "radix": 2, "bucket": 3}[args.build])
        for _ in range(3):
            g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
            _abi.msf_free(g)
        torch.cuda.synchronize(dev)
        return

    def shape_from_env():
        # sweep shape and compaction threshold from MSF_SPL / MSF_PREFETCH /
        # MSF_BPS / MSF_SWEEP / MSF_TAU (profiling runs)
        for opt, key in ((_abi.OPT_SLOTS_PER_LANE, "MSF_SPL"), (_abi.OPT_PREFETCH, "MSF_PREFETCH"),
                         (_abi.OPT_BLOCKS_PER_SM, "MSF_BPS"), (_abi.OPT_SWEEP, "MSF_SWEEP"),
                         (_abi.OPT_COMPACT_TAU, "MSF_TAU")):
            if os.environ.get(key):
                _abi.msf_set_option(opt, float(os.environ[key]))

    if args.profile_step:
        shape_from_env()
        for _ in range(2):
            g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
            _abi.msf_compute(g, mask.data_ptr(), labels.data_ptr(), total.data_ptr(), sh)
            _abi.msf_free(g)
        torch.cuda.synchronize(dev)
        return

    if args.profile_batched:
        shape_from_env()
        b = synth.workload("batch4096")
        vo, eo, G = np.ascontiguousarray(b["voff"]), np.ascontiguousarray(b["eoff"]), b["G"]
        bs, bd, bw = (torch.from_numpy(b[k]).to(dev) for k in ("src", "dst", "w"))
        bm = torch.empty(int(eo[-1]), dtype=torch.uint8, device=dev)
        bl = torch.empty(int(vo[-1]), dtype=torch.int32, device=dev)
        bt = torch.empty(G, dtype=torch.float64, device=dev)
        for _ in range(3):
            _abi.msf_compute_batched(G, vo.ctypes.data, eo.ctypes.data, bs.data_ptr(), bd.data_ptr(),
                                     bw.data_ptr(), 0, bm.data_ptr(), bl.data_ptr(), bt.data_ptr(), sh)
        torch.cuda.synchronize(dev)
        return

    if args.profile_min_edge:
        shape_from_env()
        g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
        parent = torch.arange(n, dtype=torch.int32, device=dev)
        r = torch.empty(n, dtype=torch.int64, device=dev)
        for _ in range(4):
            flush.fill_(1)
            _abi.msf_min_edge(g, parent.data_ptr(), r.data_ptr(), sh)
        torch.cuda.synchronize(dev)
        _abi.msf_free(g)
        return

    tuned = None
    if args.no_autotune:
        shape_from_env()
    else:
        from paper_2110_04865_gb300 import api, autotune
        gt = api.Graph(n, src, dst, w)
        tuned = autotune.tune(gt, use_cache=False)
        gt.free()

    # roofline of the min-edge sweep, in isolation before the timed steps:
    # every slot live (p = identity read through the gather), CUDA events
    # around the sweep launch only (msf_stats.min_edge_ms)
    g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
    gst = _abi.msf_get_stats(g)
    parent = torch.arange(n, dtype=torch.int32, device=dev)
    r = torch.empty(n, dtype=torch.int64, device=dev)
    for _ in range(3):
        _abi.msf_min_edge(g, parent.data_ptr(), r.data_ptr(), sh)
    k_times = []
    for _ in range(max(args.steps, 5)):
        flush.fill_(1)
        _abi.msf_min_edge(g, parent.data_ptr(), r.data_ptr(), sh)
        k_times.append(float(_abi.msf_get_stats(g).min_edge_ms))
    _abi.msf_free(g)
    del parent, r

    def step():
        g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
        _abi.msf_compute(g, mask.data_ptr(), labels.data_ptr(), total.data_ptr(), sh)
        st = _abi.msf_get_stats(g)
        _abi.msf_free(g)
        return st

    for _ in range(args.warmup):
        st = step()
    # kernels per step, as the library counts them (build + round loop)
    launches_per_step = int(st.kernels)

    barrier(ws)
    torch.cuda.synchronize(dev)
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    torch.cuda.synchronize(dev)
    barrier(ws)
    t_step = max_over_ranks(sum(times) / len(times), ws)
    value = ws * m / (t_step / 1e3)

    # end to end through the C ABI with pinned host buffers
    hs = torch.from_numpy(d["src"]).pin_memory()
    hd = torch.from_numpy(d["dst"]).pin_memory()
    hw = torch.from_numpy(np.ascontiguousarray(wnp)).pin_memory()
    hm = torch.empty(m, dtype=torch.uint8).pin_memory()
    hl = torch.empty(n, dtype=torch.int32).pin_memory()
    ht = torch.empty(1, dtype=torch.float64).pin_memory()

    e2e_phases = []  # (build call incl. its H2D, compute call incl. its D2H) per timed step

    def step_e2e():
        t0 = time.perf_counter()
        g = _abi.msf_build_csr(n, m, hs.data_ptr(), hd.data_ptr(), 0, hw.data_ptr(), wtype, 0, sh)
        t1 = time.perf_counter()
        _abi.msf_compute(g, hm.data_ptr(), hl.data_ptr(), ht.data_ptr(), sh)
        t2 = time.perf_counter()
        _abi.msf_free(g)
        e2e_phases.append((t1 - t0, t2 - t1))

    for _ in range(2):
        step_e2e()
    barrier(ws)
    torch.cuda.synchronize(dev)
    e2e_times = []
    e2e_phases.clear()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step_e2e()
        e2e_times.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(sum(e2e_times) / len(e2e_times), ws)
    assert float(ht[0]) == float(total.cpu()[0])

    # build / compute breakdown of one step (events around each call)
    bparts = []
    for _ in range(3):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), wtype, 0, sh)
        ev[1].record(stream)
        _abi.msf_compute(g, mask.data_ptr(), labels.data_ptr(), total.data_ptr(), sh)
        ev[2].record(stream)
        ev[2].synchronize()
        _abi.msf_free(g)
        bparts.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])))
    build_ms = statistics.median(b for b, _ in bparts)
    compute_ms = statistics.median(c for _, c in bparts)

    k_ms = statistics.median(k_times)
    alg_bytes = 16 * gst.nnz + 24 * gst.rows
    peak, peak_kind = peaks()
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "min_edge_traffic.json")
    if os.path.exists(prof):
        try:
            pj = json.load(open(prof))
            want = {k: tuned[k] for k in autotune.SHAPE_KEYS} if tuned else None
            if pj.get("workload") == args.workload and pj.get("source_hash") == build_lib.source_hash(SWEEP_SOURCES):
                for cap in pj.get("captures", []):
                    if cap.get("config") == want:
                        traffic = cap.get("dram_bytes_per_launch")
        except (ValueError, OSError, AttributeError, TypeError):
            traffic = None

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu:
        sd, sample = cpu_sample(d, args.workload)
        ms_ = len(sd["src"])
        host = host_info()
        t_or = time_oracle(sd, reps=2)
        cpu = {"value": ms_ / t_or, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": sample + ", best of 2, single thread", "host": host}
        nth = os.cpu_count() or 1
        t_mt = time_oracle(sd, reps=2, threads=nth)
        cpu_all = {"value": ms_ / t_mt, "unit": "edges/s", "cores": nth, "kind": "oracle, all cores",
                   "sample": sample + f", best of 2; the keys sorted on {nth} threads, then the same "
                             "sequential union-find scan", "host": host}
        del sd

    batched = None
    if not args.no_batched:
        batched = bench_batched(lib, dev, sh, flush, ws, rank)
    pairwise = None
    if rank == 0 and not args.no_pairwise:
        pairwise = bench_pairwise(dev, sh, flush)

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 keys (f32 weight order + edge id)", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload), "n": n, "m": m, "nnz": int(gst.nnz),
                       "rows": int(gst.rows), "rounds": int(st.rounds), "compactions": int(st.compactions),
                       "l2": "flushed before every step (256 MiB write)",
                       "build_ms": build_ms, "compute_ms": compute_ms,
                       # the same step rate without the CSR build (msf_compute alone), and the
                       # undirected edge count after the self-loops are dropped (value counts
                       # every input entry)
                       "compute_only_edges_per_s": m / (compute_ms / 1e3) if compute_ms else None,
                       "edges_without_self_loops": int(gst.nnz) // 2,
                       "min_edge_tile": ({k: tuned[k] for k in autotune.CONFIG_KEYS}
                                         if tuned else None),
                       "exec": args.exec, "builder": args.build, "kernel": args.kernel,
                       "shortcut": args.shortcut,
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "e2e": {"value": ws * m / t_e2e, "unit": "edges/s", "h2d_bytes_per_step": m * 12,
                    "d2h_bytes_per_step": m + 4 * n + 8, "ms_per_step": 1e3 * t_e2e,
                    "samples_ms": [round(1e3 * x, 2) for x in e2e_times],
                    "build_call_ms": [round(1e3 * b, 2) for b, _ in e2e_phases],
                    "compute_call_ms": [round(1e3 * c, 2) for _, c in e2e_phases]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "min-edge sweep (multilinear + projection)", "alg_bytes": alg_bytes,
                         "ms": k_ms, "alg_bytes_rule": "16 B/slot + 24 B/row",
                         "samples_ms": [round(x, 4) for x in k_times]},
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        if batched:
            line["batched_vs_looped"] = batched
        if pairwise:
            line["pairwise_vs_multilinear"] = pairwise
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_pairwise(dev, sh, flush):
    """Sec. 4.1 / Sec. 7.4 ablation on R-MAT scale 17, edge factor 8: the fused
    multilinear min-edge kernel against the pairwise formulation (a first pass
    writes p_j next to every slot, a second reduces the (a_ij, p_j) pairs).
    Per formulation: the whole round loop (msf_compute) and one full sweep
    (msf_min_edge, every slot live), best of 5 each with L2 flushed; the two
    forests must be identical."""
    import numpy as np
    import torch

    import synth
    from paper_2110_04865_gb300 import _abi
    d = synth.workload("rmat17e8")
    n, m = d["n"], len(d["src"])
    src, dst, w = (torch.from_numpy(d[k]).to(dev) for k in ("src", "dst", "w"))
    stream = torch.cuda.current_stream(dev)
    old = _abi.msf_get_option(_abi.OPT_KERNEL)
    g = _abi.msf_build_csr(n, m, src.data_ptr(), dst.data_ptr(), 0, w.data_ptr(), 0, 0, sh)
    parent = torch.arange(n, dtype=torch.int32, device=dev)
    r = torch.empty(n, dtype=torch.int64, device=dev)
    out, masks = {}, []
    try:
        for name, k in (("multilinear", 0), ("pairwise", 1)):
            _abi.msf_set_option(_abi.OPT_KERNEL, k)
            mask = torch.empty(m, dtype=torch.uint8, device=dev)
            _abi.msf_compute(g, mask.data_ptr(), 0, 0, sh)
            ct, st = [], []
            for _ in range(5):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                _abi.msf_compute(g, mask.data_ptr(), 0, 0, sh)
                b.record(stream)
                b.synchronize()
                ct.append(a.elapsed_time(b))
            _abi.msf_min_edge(g, parent.data_ptr(), r.data_ptr(), sh)
            for _ in range(5):
                flush.fill_(1)
                _abi.msf_min_edge(g, parent.data_ptr(), r.data_ptr(), sh)
                st.append(float(_abi.msf_get_stats(g).min_edge_ms))
            out[name] = {"compute_ms": min(ct), "sweep_ms": min(st)}
            masks.append(mask.cpu().numpy())
    finally:
        _abi.msf_set_option(_abi.OPT_KERNEL, old)
        _abi.msf_free(g)
    assert np.array_equal(masks[0], masks[1])
    out.update({"workload": workload_desc("rmat17e8"), "n": n, "m": m, "same_forest": True,
                "sweep_speedup": out["pairwise"]["sweep_ms"] / out["multilinear"]["sweep_ms"],
                "compute_speedup": out["pairwise"]["compute_ms"] / out["multilinear"]["compute_ms"]})
    return out


def bench_batched(lib, dev, sh, flush, ws=1, rank=0):
    """4096 graphs, n log-uniform in [64, 65536], ER or 2-D RGG, avg degree 8:
    one msf_compute_batched call vs a loop of per-graph calls.  With N ranks
    every rank takes its contiguous range of graphs (balanced by edges, no
    exchange) and the times are the slowest rank's."""
    import numpy as np
    import torch

    import synth
    from paper_2110_04865_gb300 import _abi
    from paper_2110_04865_gb300.shard import local_batch, shard_ranges
    b = synth.workload("batch4096")
    M_all, N_all, G_all = int(b["eoff"][-1]), int(b["voff"][-1]), b["G"]
    g0, g1 = shard_ranges(b["eoff"], ws)[rank]
    voff, eoff, (v0, v1), (e0, e1) = local_batch(b["voff"], b["eoff"], g0, g1)
    G = g1 - g0
    src = torch.from_numpy(b["src"][e0:e1]).to(dev)
    dst = torch.from_numpy(b["dst"][e0:e1]).to(dev)
    w = torch.from_numpy(b["w"][e0:e1]).to(dev)
    M, N = int(eoff[-1]), int(voff[-1])
    mask = torch.empty(M, dtype=torch.uint8, device=dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    totals = torch.empty(G, dtype=torch.float64, device=dev)
    vo = np.ascontiguousarray(voff)
    eo = np.ascontiguousarray(eoff)
    stream = torch.cuda.current_stream(dev)

    def batched():
        _abi.msf_compute_batched(G, vo.ctypes.data, eo.ctypes.data, src.data_ptr(), dst.data_ptr(),
                                 w.data_ptr(), 0, mask.data_ptr(), labels.data_ptr(), totals.data_ptr(), sh)

    def looped():
        for g in range(G):
            a, bb = int(eoff[g]), int(eoff[g + 1])
            nv = int(voff[g + 1] - voff[g])
            h = _abi.msf_build_csr(nv, bb - a, src.data_ptr() + 4 * a, dst.data_ptr() + 4 * a, 0,
                                   w.data_ptr() + 4 * a, 0, 0, sh)
            _abi.msf_compute(h, mask.data_ptr() + a, labels.data_ptr() + 4 * int(voff[g]),
                             totals.data_ptr() + 8 * g, sh)
            _abi.msf_free(h)

    def timed(fn, reps):
        if G == 0:
            return 0.0
        best = None
        for _ in range(reps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            bb = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            bb.record(stream)
            bb.synchronize()
            t = a.elapsed_time(bb)
            best = t if best is None else min(best, t)
        return best

    # the sweep shape and compaction threshold for this batch class, tuned on
    # the batched call itself; the loop of per-graph calls runs with the same
    # options
    from paper_2110_04865_gb300 import autotune
    saved = {k: _abi.msf_get_option(o) for k, o in (("spl", _abi.OPT_SLOTS_PER_LANE),
                                                   ("prefetch", _abi.OPT_PREFETCH),
                                                   ("blocks_per_sm", _abi.OPT_BLOCKS_PER_SM),
                                                   ("sweep", _abi.OPT_SWEEP),
                                                   ("compact_tau", _abi.OPT_COMPACT_TAU))}
    tuned = None
    if G > 0:
        tuned = autotune.tune_batched(batched, f"G{G_all}/m{M_all}", use_cache=False, device=dev)
    reps = 5
    if G > 0:
        batched()
    tb = timed(batched, reps)
    ref_tot = totals.clone()
    if G > 0:
        looped()
    tl = timed(looped, reps)
    assert torch.equal(ref_tot, totals)
    autotune.apply({k: (int(v) if k != "compact_tau" else v) for k, v in saved.items()})
    tb, tl = max_over_ranks(tb, ws), max_over_ranks(tl, ws)
    return {"graphs": G_all, "vertices": N_all, "edges": M_all, "batched_ms": tb, "looped_ms": tl,
            "speedup": tl / tb, "batched_edges_per_s": M_all / (tb / 1e3), "repeats": f"best of {reps} each",
            "tuned": ({k: tuned[k] for k in autotune.CONFIG_KEYS} if tuned else None),
            "sharding": "contiguous graph ranges balanced by edges, one per rank" if ws > 1 else "none"}


if __name__ == "__main__":
    main()
