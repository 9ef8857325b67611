#!/usr/bin/env python3
"""Throughput of per-edge AML pattern counting on B300.

One step = one aml_mine over the whole resident graph: every column of the
workload's pattern set for every edge.  Default workload: hi-small (515,088
accounts, 5,078,345 transactions over 16 days; DEG/FAN in+out, GS, SG,
CYC2..5 at 24h and 7d = 20 columns).  Prints one JSON line (rank 0), which
also carries the end-to-end time through the C ABI's host-buffer path, the
streaming latencies at three offered loads and the hi-large workload (the
largest that fits one GPU) under "large".

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun (N > 1) every rank mines its own graph of the same shape
(seed + rank): replicas, no collective on the data path; the timed region is
the max over ranks and ``value`` counts the edges of all ranks.
``--impl reference`` times the CPU oracle (edge-centric queries on a bounded
edge sample) on the host cores instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges featurized/s, all patterns, bit-exact vs plain GPU; p99 stream latency"
WORKLOAD_TEXT = {
    "hi-small": ("hi-small: 515,088 accounts, 5,078,345 transactions over 16 days, out/in-degree "
                 "Zipf(1.2) capped at 1e4, 0.1% edges in planted SG/cycle motifs; 20 columns: "
                 "DEG_OUT, DEG_IN, FAN_OUT, FAN_IN, GS, SG, CYC2..CYC5 at 24h and at 7d"),
    "tiny-10k": ("tiny-10k: 10,000 accounts, 100,000 transactions over 10 days, Zipf(1.2); "
                 "10 columns at 24h"),
    "hi-medium": ("hi-medium: 2,032,095 accounts, 31,898,238 transactions over 16 days, "
                  "out/in-degree Zipf(1.05) capped at 1e5, 0.1% edges in planted motifs; "
                  "20 columns: DEG_OUT, DEG_IN, FAN_OUT, FAN_IN, GS, SG, CYC2..CYC5 at 24h "
                  "and at 7d"),
    "hi-large": ("hi-large: 2,070,980 accounts, 179,702,229 transactions over 90 days, "
                 "Zipf(1.2) capped at 1e5, 0.05% edges in planted motifs; 10 columns: "
                 "FAN_OUT, FAN_IN, GS, SG, CYC3..CYC6 at 24h, FAN_OUT, FAN_IN at 7d"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="hi-small", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (nodes, edges, hub cap) for profiling captures")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", choices=["graph", "plain"], default="graph",
                    help="graph: the whole mine replayed as one captured CUDA graph")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help='fixed tunables instead of the autotuner, e.g. '
                         '\'{"own_max": 16, "block": 128}\' (profiling captures)')
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-fused", action="store_true",
                    help="skip timing the fused mine beside the plain one")
    ap.add_argument("--cycle-mode", choices=["auto", "plain", "fused", "persistent", "learned"],
                    default="auto", help="cycle search; auto = fastest measured")
    ap.add_argument("--cost-samples", type=int, default=1_000_000)
    ap.add_argument("--cost-epochs", type=int, default=20)
    ap.add_argument("--stream-batches", type=int, default=300,
                    help="batches per offered load (25/50/90%% of capacity)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the hi-large leg (the largest single-GPU workload)")
    ap.add_argument("--no-window-cycles", action="store_true",
                    help="skip timing the window-cycle columns (CYCW3..5 at the workload's windows)")
    ap.add_argument("--no-programs", action="store_true",
                    help="skip timing stage programs run by the generic interpreter")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    """Host-side barrier and max-reduction across ranks (gloo); no-ops at N=1."""

    def __init__(self, ws):
        self.ws = ws
        if ws > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.ws > 1:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.ws == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.ws > 1:
            self.dist.destroy_process_group()


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for i, nm in enumerate(names):
                if r[5 + i].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "of measured"
    return 6400.0, "of fallback"


# DRAM bytes per launch (read + write) from one ncu capture of hi-small at
# full size, valid only for the kernel sources it was taken with:
# KERNEL_DIGEST is the digest (kernel_digest()) of the files that define the
# measured kernels.
KERNEL_DIGEST = "d6a8f0dba9768185"
MEASURED_TRAFFIC = {"k_sg_bucket": 569.5e6, "k_cyc_level": 246.1e6, "k_sg_partition": 551.1e6,
                    "k_leg_emit": 661.5e6, "k_leg_count": 858.1e6, "k_assemble": 1256.8e6,
                    "k_fan_scan": 265.5e6, "k_fan_reduce": 143.6e6}


TRAFFIC_SOURCES = ("aml_internal.cuh", "fan.cu", "mine.cu", "mine.cuh", "pipeline.cu", "prims.cu")


def code_tokens(text: str) -> str:
    """The C/CUDA source with comments removed and whitespace runs made one
    space (string and character literals kept), so that an edit of comments
    or layout keeps the digest of the measured kernels."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_12241_b300", "csrc")
    for p in sorted(os.path.join(csrc, f) for f in TRAFFIC_SOURCES):
        h.update(os.path.relpath(p, ROOT).encode())
        with open(p, encoding="utf-8") as f:
            h.update(code_tokens(f.read()).encode())
    return h.hexdigest()[:16]


def algorithmic_bytes(kernel: str, E: int, Ev: int, pats, stats: dict) -> float:
    """Bytes per launch the kernel's definition must move (no probes, no re-reads).

    stats: the leg pass's window sizes (aml_graph_window_stats of the largest
    window with GS, SG or cycle columns: every smaller window is counted
    inside its pass): legs = temporal 2-paths, front[j] = cycle-search paths
    of j edges.  A kernel launched once per level reports the mean over its
    launches.  None for a kernel without a byte model.
      k_leg_count     per edge: src, dst, ts (12 B), its leg window's bounds and
                      leg count written (12 B); with cycle columns its closing
                      range and the range's latest edge (16 B) and the
                      cycle-capable count and bound (8 B) written; per SG/CYC
                      column one uint64 accumulator cleared (8 B); per GS
                      column the gather-side count cleared (4 B)
      k_close_range   per edge: src, dst, ts (12 B), its closing range and the
                      range's latest edge written (16 B)
      k_assemble      per edge: src, dst (8 B); per window and direction with
                      DEG/FAN columns one (DEG, FAN) pair (8 B); per GS column
                      the two leg counts (8 B); per SG/CYC column one uint64
                      accumulator (8 B); the row (4 B per column)
      k_leg_emit      per edge: src, dst, ts, leg window, leg offset (24 B); per
                      leg: the window slot (nbr, eid, t: 12 B) and its 16-B SG
                      record; per cycle-capable leg its (a, b) (8 B)
      k_sg_partition  per leg: one 16-B record read and written (32 B)
      k_sg_bucket     per leg: one 16-B record read
      k_fan_reduce    per slot: row start, t, prev (12 B), per window the DEG
                      and delta written (8 B)
      k_fan_scan      per slot: row start, eid (8 B), per window DEG and delta
                      read and (DEG, FAN) written (16 B)
      k_cyc_level     per path: the one window slot (counterparty, time: 8 B)
                      the depth-first expansion of its parent reads to reach it;
                      a launch handles one level of paths
    """
    P = len(pats)
    names = [p.name for p in pats]
    fam = [n.split("@")[0] for n in names]
    wins = {n.split("@")[1] for n in names}
    n_degfan = sum(any(f.startswith(("DEG_OUT", "FAN_OUT")) and n.endswith("@" + w)
                       for f, n in zip(fam, names)) +
                   any(f.startswith(("DEG_IN", "FAN_IN")) and n.endswith("@" + w)
                       for f, n in zip(fam, names)) for w in wins)
    n_gs = sum(f == "GS" for f in fam)
    n_acc = sum(f.startswith(("SG", "CYC")) for f in fam)
    W = sum(1 for w in wins if any(f.startswith(("DEG_OUT", "FAN_OUT")) and n.endswith("@" + w)
                                   for f, n in zip(fam, names)))
    legs = float(stats.get("legs", 0))
    front = stats.get("front", {})
    if kernel == "k_assemble":
        return E * (8 + 8 * n_degfan + 8 * n_gs + 8 * n_acc + 4 * P)
    if kernel == "k_leg_emit":
        return E * 24 + legs * (12 + 16) + front.get(2, 0) * 8
    if kernel == "k_sg_partition":
        return legs * 32
    if kernel == "k_sg_bucket":
        return legs * 16
    if kernel == "k_fan_reduce":
        return Ev * (12 + 8 * W)
    if kernel == "k_fan_scan":
        return Ev * (8 + 16 * W)
    if kernel == "k_cyc_level" and front:
        return 8.0 * sum(front.values()) / len(front)
    if kernel == "k_leg_count":
        cyc = any(f.startswith("CYC") and not f.startswith("CYCW") for f in fam)
        return E * (12 + 12 + (24 if cyc else 0) + 8 * n_acc + 4 * n_gs)
    if kernel == "k_close_range":
        return E * (12 + 16)
    return None


def time_window_cycles(graph, pats, E, use_graph, stream, flush, reps=5) -> dict:
    """Mines of the window-cycle columns (CYCW3..5 at every window of the
    workload) on the same resident graph: median of `reps` CUDA-event timed
    mines after two warm-ups, and the kernels' shares from a profiled mine."""
    import torch

    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import _lib
    from paper_2604_12241_b300 import patterns as P

    deltas = sorted({int(p.name.split("@")[1]) for p in pats})
    note = None
    while True:
        wpats = [P.window_cycle(k, d) for d in deltas for k in (3, 4, 5)]
        wps = aml.PatternSet(wpats)
        out = torch.empty((E, len(wpats)), dtype=torch.int32, device="cuda")
        try:
            for _ in range(2):
                aml.mine(graph, wps, out=out, stream=stream, use_graph=use_graph)
            torch.cuda.synchronize()
            break
        except aml.AmlError as err:   # e.g. more than 2^31 paths in the widest window
            if err.name != "AML_EUNSUPPORTED" or len(deltas) == 1:
                return {"columns": [p.name for p in wpats], "unavailable": str(err)}
            note = f"{[p.name for p in wpats]}: {err}; timed without the widest window"
            deltas = deltas[:-1]
    ts_ = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        aml.mine(graph, wps, out=out, stream=stream, use_graph=use_graph)
        b.record(stream)
        b.synchronize()
        ts_.append(a.elapsed_time(b))
    ms = float(np.median(ts_))
    _lib.profile_read(reset=True)
    _lib.profile_enable(True)
    aml.mine(graph, wps, out=out, stream=stream)
    torch.cuda.synchronize()
    _lib.profile_enable(False)
    prof = _lib.profile_read(reset=True)
    tot = sum(v[1] for v in prof.values()) or 1.0
    counts = out.cpu().numpy().view(np.uint32)
    return {"columns": [p.name for p in wpats], "ms_per_mine": ms, "edges_per_s": E / ms * 1e3,
            "instances_credited": [int(x) for x in counts.astype(np.uint64).sum(axis=0)],
            "kernels": {k: {"launches": n, "ms": round(t, 4), "share": round(t / tot, 4)}
                        for k, (n, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:6]},
            "timing": f"median of {reps} mines, CUDA events, L2 flushed between mines",
            "note": note}


def time_programs(graph, E, stream, flush, reps=3) -> dict:
    """Stage programs run by the generic interpreter on the resident graph
    (24-hour window), and one family program both ways (the family's kernels
    and the interpreter) for comparison: median of `reps` CUDA-event timed
    mines after one warm-up."""
    import torch

    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import patterns as P

    D = P.DAY
    T = P.TRIGGER

    def F(a, d, out, order, skip=0, window=P.WIN_SPAN):
        return P.Stage(P.OP_FOR_ALL, a, d, -1, 0, out, order, window, skip)

    progs = {
        # N0 -> N1 -> N2 -> N3, every hop later, within 24 hours
        "path3": P.program([T, F(1, P.DIR_OUT, 2, P.ORDER_AFTER, 0b1),
                            F(2, P.DIR_OUT, 3, P.ORDER_AFTER, 0b11)], P.AGG_INSTANCES, D),
        # common counterparties of N0 and N1 (an INTERSECT stage)
        "common_out": P.program([T, P.Stage(P.OP_INTERSECT, 0, P.DIR_OUT, 1, P.DIR_OUT, 2,
                                            P.ORDER_NONE, P.WIN_SPAN, 0b11)],
                                P.AGG_INSTANCES, D),
        # distinct senders into the trigger's later receivers (DISTINCT)
        "distinct_2hop": P.program([T, F(1, P.DIR_OUT, 2, P.ORDER_AFTER_TRIGGER, 0b1),
                                    F(2, P.DIR_IN, 3, P.ORDER_NONE, 0, P.WIN_TRAILING)],
                                   P.AGG_DISTINCT, D),
        "GS@86400 interpreted": P.interpreted(P.gather_scatter(D)),
        "GS@86400 family kernels": P.gather_scatter(D),
        "CYC3@86400 interpreted": P.interpreted(P.cycle(3, D)),
        "CYC3@86400 family kernels": P.cycle(3, D),
    }
    res = {}
    out = torch.empty((E, 1), dtype=torch.int32, device="cuda")
    for name, pat in progs.items():
        ps = aml.PatternSet([pat])
        try:
            aml.mine(graph, ps, out=out, stream=stream)
            torch.cuda.synchronize()
        except aml.AmlError as err:
            res[name] = {"unavailable": str(err)}
            continue
        ts_ = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            aml.mine(graph, ps, out=out, stream=stream)
            b.record(stream)
            b.synchronize()
            ts_.append(a.elapsed_time(b))
        ms = float(np.median(ts_))
        total = int(out.cpu().numpy().view(np.uint32).astype(np.uint64).sum())
        res[name] = {"column": ps.columns[0]["name"], "ms_per_mine": round(ms, 3),
                     "edges_per_s": E / ms * 1e3, "sum_of_counts": total}
    return {"programs": res, "timing": f"median of {reps} mines, CUDA events, L2 flushed "
            "between mines; one column per mine, plain launches"}


# --------------------------------------------------------------- reference

def run_reference(args, ws, rank):
    """The CPU oracle, as it stands, on the host cores (edge-centric queries)."""
    if rank != 0:
        return
    import oracle
    from paper_2604_12241_b300 import patterns as P
    g = make_workload(args, rank)
    pats = P.workload_patterns(args.workload)
    cols = oracle.columns_from_names([p.name for p in pats])
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    # calibrate the per-step sample so the whole run stays within minutes
    probe = rng.choice(g.n_edges, 2000, replace=False)
    t0 = time.perf_counter()
    og.count_edges(cols, probe, threads=cores)
    per_edge = (time.perf_counter() - t0) / probe.size
    budget = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    n = int(min(g.n_edges, max(1000, budget / max(per_edge, 1e-9))))
    for _ in range(args.warmup):
        og.count_edges(cols, rng.choice(g.n_edges, n, replace=False), threads=cores)
    t = 0.0
    for _ in range(args.steps):
        ids = rng.choice(g.n_edges, n, replace=False)
        t0 = time.perf_counter()
        og.count_edges(cols, ids, threads=cores)
        t += time.perf_counter() - t0
    value = n * args.steps / t
    sample = (f"edge-centric oracle queries of {n} uniformly sampled edges per step "
              f"({len(cols)} columns each) of {args.workload}")
    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(args.workload, g, len(cols), args.scale, ws),
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores,
                             "kind": "oracle", "sample": sample, "sample_edges_per_step": n},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(g, pats, seconds: float) -> dict:
    import oracle
    from paper_2604_12241_b300 import patterns as P
    cols = oracle.columns_from_names([p.name for p in pats])
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(3)
    probe = rng.choice(g.n_edges, 2000, replace=False)
    t0 = time.perf_counter()
    og.count_edges(cols, probe, threads=cores)
    per_edge = (time.perf_counter() - t0) / probe.size
    n = int(min(g.n_edges, max(2000, seconds / max(per_edge, 1e-9))))
    ids = rng.choice(g.n_edges, n, replace=False)
    t0 = time.perf_counter()
    og.count_edges(cols, ids, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "edges/s", "cores": cores, "kind": "oracle",
            "sample": f"edge-centric oracle queries of {n} uniformly sampled edges "
                      f"({len(cols)} columns each), {dt:.1f} s on {cores} threads"}


# ---------------------------------------------------------------- streaming

STREAM_DAYS = 31        # the stream's graph: hi-medium's shape and daily rate, 31 days
STREAM_PRE_DAYS = 9     # appended untimed before the measured batches
STREAM_LOADS = (0.25, 0.5, 0.9)


def run_stream(args, rank) -> dict:
    """Streaming serving (the fifth workload): a HI-Medium-shaped graph
    (2,032,095 accounts, Zipf 1.05, hubs to 1e5) at HI-Medium's rate of
    about 2M transactions a day, generated over 31 days so that enough
    batches arrive; 20 columns, a 7-day resident window.  The first 9 days
    are appended in 2M-edge batches (untimed).  Then batches of log-uniform
    size in [1e3, 1e5] arrive: first back to back (service time, capacity),
    then as Poisson processes offered at 25%, 50% and 90% of the measured
    capacity (latency = queueing + service), ``--stream-batches`` batches at
    each load, served one batch per append and again with the queued
    batches merged into one append."""
    import aml_synth
    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import patterns as P
    params = dict(aml_synth.WORKLOADS["hi-medium"])
    params["n_edges"] = int(params["n_edges"] * STREAM_DAYS / params["days"])
    params["days"] = STREAM_DAYS
    params["seed"] = 20260005 + rank * 1000
    g = aml_synth.generate(name="stream", **params)
    pats = P.workload_patterns("hi-medium")
    ps = aml.PatternSet(pats)
    st = aml.Stream(ps, g.n_nodes, resident_window=7 * P.DAY, mem_budget=96 << 30)
    pos = 0
    t_pre = int(np.searchsorted(g.ts, STREAM_PRE_DAYS * P.DAY))
    while pos < t_pre:
        n = min(2_000_000, t_pre - pos)
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n], g.amount[pos:pos + n])
        pos += n
    rng = np.random.default_rng(20260005)

    def next_batch():
        nonlocal pos
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
        n = min(n, g.n_edges - pos)
        b = (g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n], g.amount[pos:pos + n])
        pos += n
        return b

    service, sizes = [], []
    for _ in range(max(30, args.stream_batches // 3)):
        if pos >= g.n_edges:
            break
        b = next_batch()
        t0 = time.perf_counter()
        st.append(*b)
        service.append(time.perf_counter() - t0)
        sizes.append(len(b[0]))
    cap_eps = sum(sizes) / sum(service)               # edges/s, back to back
    mean_n = float(np.mean(sizes))
    ms = lambda v, q: float(np.percentile(np.asarray(v) * 1e3, q)) if v else None
    # Offered loads.  A batch's latency runs from its arrival to the end of
    # the append that holds it.  "one batch per append" serves the queue in
    # arrival order; "queued batches merged" appends, whenever the server
    # is free, every batch that has arrived by then as one (consecutive
    # batches are one time-ordered slice), so a burst costs one recount
    # instead of one per batch.  Counts are the same either way.
    def serve(load, merge):
        lam = load * cap_eps / mean_n                 # batches/s
        arr, sl = [], []
        t = 0.0
        for _ in range(args.stream_batches):
            if pos >= g.n_edges:
                break
            t += rng.exponential(1.0 / lam)
            lo = pos
            b = next_batch()
            arr.append(t)
            sl.append((lo, lo + len(b[0])))
        lat, appends = [], 0
        t_start = time.perf_counter()
        k = 0
        while k < len(arr):
            now = time.perf_counter() - t_start
            if now < arr[k]:
                time.sleep(arr[k] - now)
                now = time.perf_counter() - t_start
            j = k + 1
            while merge and j < len(arr) and arr[j] <= now:
                j += 1
            lo, hi = sl[k][0], sl[j - 1][1]
            st.append(g.src[lo:hi], g.dst[lo:hi], g.ts[lo:hi], g.amount[lo:hi])
            done = time.perf_counter() - t_start
            lat.extend(done - a for a in arr[k:j])
            appends += 1
            k = j
        span = time.perf_counter() - t_start
        return {"batches": len(lat), "appends": appends, "p50_ms": ms(lat, 50),
                "p99_ms": ms(lat, 99), "max_ms": ms(lat, 100),
                "edges_per_s": (sl[-1][1] - sl[0][0]) / span if lat else None,
                "arrivals": "Poisson, batches/s = %.2f" % lam}

    loads = {}
    for load in STREAM_LOADS:
        one = serve(load, False)
        loads[f"load_{int(round(load * 100))}pct"] = dict(one, merged=serve(load, True))
    info = st.info()
    st.close()
    return {"workload": ("hi-medium shape (2,032,095 accounts, Zipf 1.05, hubs to 1e5) at "
                         "~2.0M transactions/day over 31 days; 7-day resident window, 20 columns"),
            "resident_rows": info["resident_rows"], "batches": len(service) + sum(
                v["batches"] + v["merged"]["batches"] for v in loads.values()),
            "batch_edges": "log-uniform in [1e3, 1e5]",
            "service_batches": len(service),
            "service_ms_p50": ms(service, 50), "service_ms_p99": ms(service, 99),
            "capacity_edges_per_s": cap_eps, **loads,
            "method": "exact: one mine of the window W within 7d of the batch plus the batch, "
                      "counting only instances whose latest edge is new"}


# ------------------------------------------------------------ end to end

def time_e2e(args, g, ps, E, Pn, ref_out, ws, dist) -> dict:
    """End to end through the C ABI with host buffers, every step: the
    step's transactions from page-locked host arrays (aml_graph_create with
    AML_PTR_HOST: the library copies them to the device and builds the
    graph), the mine, and the counts back into page-locked host memory
    (aml_mine with AML_MINE_HOST_OUTPUT | AML_MINE_HOST_ASYNC).  Steps use a
    ring of three slots (stream + output buffer); a step takes its slot by
    destroying the slot's previous graph, which waits for that step's copy
    back.  aml_graph_create waits for its build and the first mine of a graph
    waits once for its sizes, so two pipelines are timed: one host thread
    (the next step's upload and build overlap this step's copy back), and
    two host threads (the calls release the GIL), reporting the faster."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import paper_2604_12241_b300 as aml
    R = 3
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
           (("src", g.src), ("dst", g.dst), ("ts", g.ts), ("amount", g.amount))}
    host = {k: t.numpy() for k, t in pin.items()}
    S = [torch.cuda.Stream() for _ in range(R)]
    out_pin = [torch.empty((E, Pn), dtype=torch.int32).pin_memory() for _ in range(R)]
    out_host = [t.numpy().view(np.uint32) for t in out_pin]
    live = [None] * R
    slot_lock = [threading.Lock() for _ in range(R)]
    dev = torch.cuda.current_device()

    def take_slot(i):
        if live[i] is not None:
            live[i].close()
            live[i] = None

    def step(k):
        torch.cuda.set_device(dev)  # worker threads start on device 0
        i = k % R
        with slot_lock[i]:
            take_slot(i)
            gg = aml.Graph(host["src"], host["dst"], host["ts"], g.n_nodes,
                           amount=host["amount"], assume_sorted=True, stream=S[i])
            aml.mine(gg, ps, out=out_host[i], stream=S[i], host_output=True, host_async=True)
            live[i] = gg

    def run(n_steps, workers):
        if workers == 1:
            for k in range(n_steps):
                step(k)
        else:
            with ThreadPoolExecutor(max_workers=workers) as pool:
                for f in [pool.submit(step, k) for k in range(n_steps)]:
                    f.result()
        for i in range(R):
            take_slot(i)

    times = {}
    for workers in (1, 2):
        run(R, workers)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(args.e2e_steps, workers)
        torch.cuda.synchronize()
        times[workers] = dist.max(time.perf_counter() - t0)
    host_threads = min(times, key=times.get)
    e2e_s = times[host_threads]
    last = out_host[(args.e2e_steps - 1) % R]
    return {"value": ws * E * args.e2e_steps / e2e_s, "unit": "edges/s",
            "h2d_bytes_per_step": int(E * 16), "d2h_bytes_per_step": int(E * Pn * 4),
            "steps": args.e2e_steps, "ms_per_step": 1000.0 * e2e_s / args.e2e_steps,
            "matches_device_output": bool(np.array_equal(
                last, ref_out.cpu().numpy().view(np.uint32))),
            "host_threads": host_threads,
            "ms_per_step_by_host_threads": {str(w): round(1000.0 * t / args.e2e_steps, 3)
                                            for w, t in times.items()},
            "api": "aml_graph_create(AML_PTR_HOST | AML_ASSUME_SORTED) + aml_mine("
                   "AML_MINE_HOST_OUTPUT | AML_MINE_HOST_ASYNC), page-locked host buffers",
            "includes": "host inputs -> device, graph build, mine, counts -> host memory, "
                        "every step; steps over a ring of three streams"}


# ------------------------------------------------------------ shared timing

def mine_ms(graph, ps, out, stream, flush, use_graph, mode, reps) -> float:
    """Median CUDA-event time of `reps` mines (L2 flushed before each, two
    untimed mines first)."""
    import torch

    import paper_2604_12241_b300 as aml
    for _ in range(2):
        aml.mine(graph, ps, out=out, stream=stream, use_graph=use_graph, mode=mode)
    torch.cuda.synchronize()
    ts_ = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        aml.mine(graph, ps, out=out, stream=stream, use_graph=use_graph, mode=mode)
        b.record(stream)
        b.synchronize()
        ts_.append(a.elapsed_time(b))
    return float(np.median(ts_))


def profiled_mines(graph, ps, out, stream, flush, mode, n) -> tuple:
    """Per-kernel CUDA-event times of n plain (not replayed) mines: the
    library records a pair of events around every launch on its stream."""
    import torch

    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import _lib
    torch.cuda.synchronize()
    _lib.profile_read(reset=True)
    _lib.profile_enable(True)
    total = 0.0
    for _ in range(n):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        aml.mine(graph, ps, out=out, stream=stream, mode=mode)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    _lib.profile_enable(False)
    return total, _lib.profile_read(reset=True)


def leg_pass_window(pats) -> int:
    """The window whose leg pass counts every GS, SG and cycle column (the
    largest such window; the smaller ones are counted inside its pass), or
    the largest window when no column needs legs."""
    fam_of = [(p.name.split("@")[0], int(p.name.split("@")[1])) for p in pats]
    legs = [d for f, d in fam_of
            if f == "GS" or f.startswith("SG") or (f.startswith("CYC") and not f.startswith("CYCW"))]
    return max(legs) if legs else max(d for _, d in fam_of)


def roofline_of(prof, total_ms, graph, pats, E, Ev) -> dict:
    """The dominant kernel's HBM roofline: algorithmic bytes per launch over
    its mean launch time (CUDA events), against the measured copy
    bandwidth."""
    dom_name, (dom_n, dom_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    big = leg_pass_window(pats)
    ws_stats = graph.window_stats(big)
    stats = {"legs": ws_stats["n_legs"], "front": ws_stats["n_front"]}
    peak, peak_src = measured_peak()
    alg = algorithmic_bytes(dom_name, E, Ev, pats, stats)
    achieved = alg / (dom_ms / dom_n / 1000.0) / 1e9 if alg is not None else None
    return {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "peak_source": peak_src, "launch_ms": dom_ms / dom_n,
            "share_of_step": dom_ms / total_ms, "algorithmic_bytes_per_launch": alg,
            "timed_in": "plain-mode profiled pass (CUDA events per launch)",
            "leg_pass": {"delta": big, **stats}}


# --------------------------------------------------------------- hi-large

def run_large(args, rank, local) -> dict:
    """The largest single-GPU workload (hi-large: 2,070,980 accounts,
    179,702,229 transactions over 90 days; FAN_OUT, FAN_IN, GS, SG,
    CYC3..CYC6 at 24h, FAN_OUT, FAN_IN at 7d): the resident graph mined with
    graph replay after autotuning, with the cost model trained for learned
    binning; level-by-level and learned-binned cycle searches both timed."""
    import torch

    import aml_synth
    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import patterns as P
    params = dict(aml_synth.WORKLOADS["hi-large"])
    params["seed"] += rank * 1000
    g = aml_synth.generate(name="hi-large", **params)
    pats = P.workload_patterns("hi-large")
    E, Pn = g.n_edges, len(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount, assume_sorted=True)
    Ev = graph.info()["n_list_edges"]
    ps = aml.PatternSet(pats)
    out = torch.empty((E, Pn), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    best, best_ms = aml.autotune(graph, ps, repeats=3)
    rep = aml.cost_train(graph, ps, max_samples=args.cost_samples, epochs=args.cost_epochs,
                         seed=20260004)
    modes = {}
    clocks = ClockSampler(local)
    clocks.start()
    for m in ("plain", "fused", "learned"):
        modes[m] = mine_ms(graph, ps, out, stream, flush, True, m, 5)
    clk = clocks.stop()
    mode = min(modes, key=modes.get)
    plain = out.clone()
    aml.mine(graph, ps, out=out, stream=stream, use_graph=True, mode="learned")
    same = bool(torch.equal(out, plain))
    total, prof = profiled_mines(graph, ps, out, stream, flush, mode, 1)
    res = {"workload": WORKLOAD_TEXT["hi-large"], "n_edges": E, "columns": Pn,
           "ms_per_mine": modes[mode], "edges_per_s": E / modes[mode] * 1e3,
           "cycle_mode": mode, "cycle_modes_ms": modes, "replay": "one CUDA graph per mine",
           "learned_equals_plain": same,
           "cost_model": {k: rep[k] for k in ("n_train", "n_test", "test_log_mae",
                                                "test_spearman", "degree_spearman")},
           "autotune": {"tuning": best, "best_ms": best_ms},
           "roofline": roofline_of(prof, total, graph, pats, E, Ev),
           "kernels": {k: {"launches": n, "ms": round(t, 4), "share": round(t / total, 4)}
                       for k, (n, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]},
           "clocks": clk,
           "timing": "median of 5 replayed mines per mode, CUDA events, L2 flushed between"}
    del out, plain, flush
    graph.close()
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------------- ours

def workload_config(name: str, g, n_cols: int, scale: float, ws: int) -> dict:
    """The static description of the timed workload (both arms print it)."""
    return {"workload": WORKLOAD_TEXT[name], "n_edges": int(g.n_edges), "n_nodes": int(g.n_nodes),
            "columns": n_cols, "scale": scale,
            "l2": "flushed between steps (256 MB write, untimed)",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def run_ours(args, ws, rank, local):
    import torch

    import aml_synth
    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import _lib
    from paper_2604_12241_b300 import patterns as P

    torch.cuda.set_device(local)
    dist = Dist(ws)
    g = make_workload(args, rank)
    pats = P.workload_patterns(args.workload)
    E, Pn = g.n_edges, len(pats)

    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount, assume_sorted=True)
    ps = aml.PatternSet(pats)
    out = torch.empty((E, Pn), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    stream = torch.cuda.current_stream()

    tune_info = None
    if args.tuning:
        graph.set_tuning(**json.loads(args.tuning))
        tune_info = {"tuning": graph.tuning(), "fixed": True}
    elif not args.no_autotune:
        t0 = time.perf_counter()
        best, best_ms = aml.autotune(graph, ps, repeats=3)
        tune_info = {"tuning": best, "best_ms": best_ms, "seconds": time.perf_counter() - t0}
    use_graph = args.mode == "graph"
    # cost model for learned binning, then each cycle-search mode timed
    cost_report = None
    if args.cycle_mode in ("auto", "learned"):
        cost_report = aml.cost_train(graph, ps, max_samples=args.cost_samples,
                                     epochs=args.cost_epochs, seed=20260003)
    modes = {}
    if args.cycle_mode == "auto":
        for m in ("plain", "fused", "persistent", "learned"):
            modes[m] = mine_ms(graph, ps, out, stream, flush, use_graph, m, 10)
        cycle_mode = min(modes, key=modes.get)
    else:
        cycle_mode = args.cycle_mode
        if cycle_mode == "plain" and not args.no_fused:  # the fused mine beside it
            for m in ("plain", "fused"):
                modes[m] = mine_ms(graph, ps, out, stream, flush, use_graph, m, 10)
    for _ in range(max(3, args.warmup)):
        aml.mine(graph, ps, out=out, use_graph=use_graph, mode=cycle_mode)
    torch.cuda.synchronize()
    graph.sync()

    # headline: the chosen mode, clocks sampled during the timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    l0 = _lib.launch_count()
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                     # evict L2 between steps (not timed)
        ev[k][0].record(stream)
        aml.mine(graph, ps, out=out, stream=stream, use_graph=use_graph, mode=cycle_mode)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    dist.barrier()
    launches = _lib.launch_count() - l0
    clk = clocks.stop()
    graph.sync()
    dev_ms_max = dist.max(sum(a.elapsed_time(b) for a, b in ev))
    # per-kernel CUDA-event times come from plain (not replayed) mines:
    # events cannot be recorded between the kernels of a replayed graph
    prof_steps = max(3, min(args.steps, 10))
    plain_ms, prof = profiled_mines(graph, ps, out, stream, flush, cycle_mode, prof_steps)

    e2e = None if args.no_e2e else time_e2e(args, g, ps, E, Pn, out, ws, dist)

    line = None
    if rank == 0:
        value = ws * E * args.steps / (dev_ms_max / 1000.0)
        info = graph.info()
        roof = roofline_of(prof, plain_ms, graph, pats, E, info["n_list_edges"])
        traffic = None
        if (args.workload == "hi-small" and args.scale == 1.0
                and kernel_digest() == KERNEL_DIGEST):
            traffic = MEASURED_TRAFFIC.get(roof["kernel"])
        roof["traffic"] = traffic
        roof["traffic_unit"] = "DRAM bytes read + written per launch (ncu, full size)"
        kernels = {k: {"launches": n, "ms_per_step": round(ms / prof_steps, 4),
                       "share": round(ms / plain_ms, 4)}
                   for k, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws,
                "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "impl": "ours",
                "config": workload_config(args.workload, g, Pn, args.scale, ws),
                "run": {"mode": args.mode, "autotune": tune_info, "cycle_mode": cycle_mode,
                        "cycle_modes_ms": modes or None, "wall_s_timed_loop": wall},
                "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "clocks": clk,
                "plain_ms_per_step": plain_ms / prof_steps,
                "cost_model": cost_report,
                "kernels": kernels}
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, pats, args.cpu_seconds)
        if not args.no_window_cycles:
            line["window_cycles"] = time_window_cycles(graph, pats, E, use_graph, stream, flush)
        if not args.no_programs:
            line["interpreter"] = time_programs(graph, E, stream, flush)
    del out, flush
    graph.close()
    torch.cuda.empty_cache()
    if not args.no_stream:
        st = run_stream(args, rank)
        if line is not None:
            line["stream"] = st
            # the serving loop merges queued batches; one append per batch beside it
            line["p99_stream_latency_ms"] = st["load_50pct"]["merged"]["p99_ms"]
            line["p99_stream_latency_ms_one_per_append"] = st["load_50pct"]["p99_ms"]
    if not args.no_large and args.workload != "hi-large":
        large = run_large(args, rank, local)
        if line is not None:
            line["large"] = large
    dist.close()
    if line is not None:
        print(json.dumps(line), flush=True)


def make_workload(args, rank):
    import aml_synth
    params = dict(aml_synth.WORKLOADS[args.workload])
    if args.scale != 1.0:
        params["n_nodes"] = max(1000, int(params["n_nodes"] * args.scale))
        params["n_edges"] = max(10_000, int(params["n_edges"] * args.scale))
        if params.get("d_max"):
            params["d_max"] = max(50.0, params["d_max"] * args.scale)
    params["seed"] += rank * 1000     # independent replica per rank
    return aml_synth.generate(name=args.workload, **params)


def main():
    args = parse()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
