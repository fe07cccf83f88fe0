"""Autotuner for the min-edge sweep's tile shape and the compaction threshold.

For a built graph it times the whole round loop (msf_compute), or one sweep
(msf_min_edge with p = identity, every slot live), for every combination of
sweep form
(register tiles, with or without next-tile prefetch; the shared-memory
pipeline; the register pipeline), slots per lane (tile width 32*V) and
resident blocks per SM,
keeps the fastest, and sets it as the library's process-wide option; with
the round-loop objective it then times the compaction thresholds in
TAU_CANDIDATES with that shape (compaction pays only when enough rounds
follow on a much smaller edge list).  Durations
come from the library itself (CUDA events around the sweep launch only,
``msf_stats.min_edge_ms``).  Results are cached per device and graph class
(log2 of the slot count, rounded average degree) in
``_build/autotune.json`` next to the library.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import torch

from . import _abi

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
# (slots per lane, prefetch, blocks per SM, sweep form)
CANDIDATES = ([(spl, pf, bps, 0) for spl in (4, 8, 16) for pf in (0, 1) for bps in (2, 4, 8)]
              + [(spl, 0, bps, 1) for spl in (4, 8, 16) for bps in (1, 2, 3, 4)]
              + [(spl, 0, bps, 2) for spl in (4, 8) for bps in (2, 3, 4)])
SHAPE_KEYS = ("spl", "prefetch", "blocks_per_sm", "sweep")
CONFIG_KEYS = SHAPE_KEYS + ("compact_tau",)
# compaction thresholds, the library's default first (kept on near-ties)
TAU_CANDIDATES = (0.5, 0.25, 0.0)


def pick_shape(table):
    """The shape to keep from rows (ms, sweep_ms, spl, prefetch, blocks_per_sm,
    sweep): the fastest by ms; among the rows within 1 % of it (closer than
    the measurements' noise), the one whose full sweep is fastest."""
    fastest = min(t[0] for t in table)
    return min((t for t in table if t[0] <= 1.01 * fastest), key=lambda t: t[1])


def pick_first(rows):
    """The first row, in candidate order, whose time (its first field) is
    within 1 % of the fastest: an earlier candidate wins a near-tie (for the
    compaction thresholds the library's default comes first)."""
    fastest = min(r[0] for r in rows)
    return next(r for r in rows if r[0] <= 1.01 * fastest)


def _key(device: torch.device, st) -> str:
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    cls = int(round(math.log2(max(int(st.nnz), 1))))
    deg = int(round(st.nnz / max(int(st.rows), 1)))
    deg_cls = int(round(math.log2(max(deg, 1))))
    return f"{name}/nnz2^{cls}/deg2^{deg_cls}"


def _load_cache() -> dict:
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def apply(cfg: dict):
    _abi.msf_set_option(_abi.OPT_SLOTS_PER_LANE, cfg["spl"])
    _abi.msf_set_option(_abi.OPT_PREFETCH, cfg["prefetch"])
    _abi.msf_set_option(_abi.OPT_BLOCKS_PER_SM, cfg["blocks_per_sm"])
    _abi.msf_set_option(_abi.OPT_SWEEP, cfg.get("sweep", 0))
    if "compact_tau" in cfg:
        _abi.msf_set_option(_abi.OPT_COMPACT_TAU, cfg["compact_tau"])


def tune(graph, reps: int = 5, use_cache: bool = True, flush_bytes: int = 256 << 20,
         objective: str = "compute") -> dict:
    """Times every candidate on `graph` (an api.Graph) and applies the fastest.
    objective "compute": the whole round loop (msf_compute, edge mask only;
    later rounds, where parents repeat, weigh in); "sweep": one min-edge
    sweep with every slot live.  Returns dict(spl, prefetch, blocks_per_sm,
    sweep, ms, table)."""
    dev = graph.device if graph.device is not None else torch.device("cuda", torch.cuda.current_device())
    st = graph.stats()
    key = _key(dev, st) + f"/{objective}"
    cache = _load_cache()
    if use_cache and key in cache:
        apply(cache[key])
        return dict(cache[key], cached=True)
    parent = torch.arange(graph.n, dtype=torch.int32, device=dev)
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    table = []
    for spl, pf, bps, sw in CANDIDATES:
        apply(dict(spl=spl, prefetch=pf, blocks_per_sm=bps, sweep=sw))
        ctimes, stimes = [], []
        if objective == "compute":
            graph.compute(mask=True, labels=False, total=False)  # warm-up (and graph instantiation)
            for _ in range(max(reps, 3)):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                graph.compute(mask=True, labels=False, total=False)
                b.record(stream)
                b.synchronize()
                ctimes.append(a.elapsed_time(b))
        graph.min_edge(parent)  # warm-up
        for _ in range(reps):
            flush.fill_(1)
            graph.min_edge(parent)
            stimes.append(float(graph.stats().min_edge_ms))
        sweep_ms = statistics.median(stimes)
        ms = statistics.median(ctimes) if ctimes else sweep_ms
        table.append((ms, sweep_ms, spl, pf, bps, sw))
    ms, sweep_ms, spl, pf, bps, sw = pick_shape(table)
    best = dict(spl=spl, prefetch=pf, blocks_per_sm=bps, sweep=sw, ms=ms, sweep_ms=sweep_ms)
    if objective == "compute":
        # the compaction threshold with that shape; an earlier candidate wins
        # a near-tie
        ttimes = []
        for tau in TAU_CANDIDATES:
            apply(dict(best, compact_tau=tau))
            graph.compute(mask=True, labels=False, total=False)
            ct = []
            for _ in range(max(reps, 3)):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                graph.compute(mask=True, labels=False, total=False)
                b.record(stream)
                b.synchronize()
                ct.append(a.elapsed_time(b))
            ttimes.append((statistics.median(ct), tau))
        t_ms, tau = pick_first(ttimes)
        best.update(compact_tau=tau, ms=t_ms)
    else:
        best.update(compact_tau=_abi.msf_get_option(_abi.OPT_COMPACT_TAU))
    apply(best)
    cache[key] = best
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    except OSError:
        pass
    return dict(best, cached=False,
                table=[dict(ms=t, sweep_ms=u, spl=a, prefetch=b, blocks_per_sm=c, sweep=e)
                       for t, u, a, b, c, e in table])


def tune_batched(call, key: str, reps: int = 3, use_cache: bool = True, flush_bytes: int = 256 << 20,
                 device=None) -> dict:
    """The same search for the batched form: `call()` enqueues one
    msf_compute_batched call on the current stream (the whole batch: build
    and round loop); every sweep shape is timed on it, then the compaction
    thresholds with the fastest shape.  `key` names the batch class for the
    cache.  Returns dict(spl, prefetch, blocks_per_sm, sweep, compact_tau, ms)."""
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    name = torch.cuda.get_device_name(dev).replace(" ", "_")
    ckey = f"{name}/batched/{key}"
    cache = _load_cache()
    if use_cache and ckey in cache:
        apply(cache[ckey])
        return dict(cache[ckey], cached=True)
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed():
        call()  # warm-up (and graph instantiation for a new shape)
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    tau0 = _abi.msf_get_option(_abi.OPT_COMPACT_TAU)
    table = []
    for spl, pf, bps, sw in CANDIDATES:
        apply(dict(spl=spl, prefetch=pf, blocks_per_sm=bps, sweep=sw, compact_tau=tau0))
        table.append((timed(), spl, pf, bps, sw))
    ms, spl, pf, bps, sw = pick_first(table)
    best = dict(spl=spl, prefetch=pf, blocks_per_sm=bps, sweep=sw)
    ttimes = []
    for tau in TAU_CANDIDATES:
        apply(dict(best, compact_tau=tau))
        ttimes.append((timed(), tau))
    t_ms, tau = pick_first(ttimes)
    best.update(compact_tau=tau, ms=t_ms)
    apply(best)
    cache[ckey] = best
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    except OSError:
        pass
    return dict(best, cached=False)
