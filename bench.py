#!/usr/bin/env python3
"""Throughput of per-edge AML pattern counting on B300.

One step = one aml_mine over the whole resident graph: every column of the
workload's pattern set for every edge.  Default workload: hi-small (515,088
accounts, 5,078,345 transactions over 16 days; DEG/FAN in+out, GS, SG,
CYC2..5 at 24h and 7d = 20 columns).  Prints one JSON line (rank 0).

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
    ap.add_argument("--cycle-mode", choices=["auto", "plain", "persistent", "learned"],
                    default="auto", help="cycle search; auto = fastest measured")
    ap.add_argument("--cost-samples", type=int, default=1_000_000)
    ap.add_argument("--cost-epochs", type=int, default=20)
    ap.add_argument("--stream-batches", type=int, default=30)
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
# full size (profiles/dram_hi_small.md), valid only for the kernel sources it
# was taken with: KERNEL_DIGEST is the digest (kernel_digest()) of the files
# that define the measured kernels.
KERNEL_DIGEST = "c5d6358914ba8ac2"
MEASURED_TRAFFIC = {"k_cyc_level": 267.0e6, "k_sg_bucket": 519.2e6, "k_leg_emit": 610.1e6,
                    "k_sg_partition": 548.5e6, "k_fan_reduce": 230.5e6, "k_fan_scan": 314.4e6,
                    "k_assemble": 1076.7e6, "k_leg_count": 698.2e6}


TRAFFIC_SOURCES = ("aml_internal.cuh", "fan.cu", "mine.cu", "mine.cuh", "pipeline.cu", "prims.cu")


def kernel_digest() -> str:
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_12241_b300", "csrc")
    for p in sorted(os.path.join(csrc, f) for f in TRAFFIC_SOURCES):
        h.update(os.path.relpath(p, ROOT).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def algorithmic_bytes(kernel: str, E: int, Ev: int, pats, stats: dict) -> float:
    """Bytes per launch the kernel's definition must move (no probes, no re-reads).

    stats: the leg pass's window sizes (aml_graph_window_stats of the largest
    window: every smaller window is counted inside its pass): legs = temporal
    2-paths, front[j] = cycle-search paths of j edges.  A kernel launched once
    per level reports the mean over its launches.
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
      k_cyc_level     per path: its parent link and slot (8 B), its anchor's
                      closing range (8 B), its next-hop count and start (8 B)
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
        return 24.0 * sum(front.values()) / len(front)
    return float("nan")


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
    import aml_synth
    import oracle
    from paper_2604_12241_b300 import patterns as P
    g = aml_synth.workload(args.workload)
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
            "config": {"workload": WORKLOAD_TEXT[args.workload], "n_edges": g.n_edges,
                       "n_nodes": g.n_nodes, "columns": len(cols), "sample_edges": n},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
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

def run_stream(args, rank) -> dict:
    """Streaming serving (the fifth workload): a HI-Medium-shaped graph (2,032,095
    accounts, 31,898,238 transactions over 16 days), 20 columns, a 7-day
    resident window.  The first 9 days are appended in 2M-edge batches
    (untimed); then batches of log-uniform size in [1e3, 1e5] arrive, first
    back to back (service latency), then as a Poisson process offered at 50%
    of the measured capacity (latency = queueing + service)."""
    import aml_synth
    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import patterns as P
    params = dict(aml_synth.WORKLOADS["hi-medium"])
    params["seed"] += rank * 1000
    g = aml_synth.generate(name="hi-medium", **params)
    pats = P.workload_patterns("hi-medium")
    ps = aml.PatternSet(pats)
    st = aml.Stream(ps, g.n_nodes, resident_window=7 * P.DAY, mem_budget=96 << 30)
    pos = 0
    t_pre = int(np.searchsorted(g.ts, 9 * P.DAY))
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
    for _ in range(args.stream_batches):
        if pos >= g.n_edges:
            break
        b = next_batch()
        t0 = time.perf_counter()
        st.append(*b)
        service.append(time.perf_counter() - t0)
        sizes.append(len(b[0]))
    cap_eps = sum(sizes) / sum(service)               # edges/s, back to back
    mean_n = float(np.mean(sizes))
    lam = 0.5 * cap_eps / mean_n                      # batches/s at 50% load
    lat, t_next, sizes2 = [], time.perf_counter(), []
    for _ in range(args.stream_batches):
        if pos >= g.n_edges:
            break
        t_next += rng.exponential(1.0 / lam)
        b = next_batch()
        now = time.perf_counter()
        if now < t_next:
            time.sleep(t_next - now)
        st.append(*b)
        lat.append(time.perf_counter() - t_next)
        sizes2.append(len(b[0]))
    info = st.info()
    st.close()
    ms = lambda v, q: float(np.percentile(np.asarray(v) * 1e3, q)) if v else None
    return {"workload": "hi-medium shape, 7-day resident window, 20 columns",
            "resident_rows": info["resident_rows"], "batches": len(service) + len(lat),
            "batch_edges": "log-uniform in [1e3, 1e5]",
            "service_ms_p50": ms(service, 50), "service_ms_p99": ms(service, 99),
            "capacity_edges_per_s": cap_eps,
            "load_50pct": {"p50_ms": ms(lat, 50), "p99_ms": ms(lat, 99),
                           "edges_per_s": sum(sizes2) / (sum(lat) if lat else 1),
                           "arrivals": "Poisson, batches/s = %.2f" % lam},
            "method": "exact: one mine of the window W within 7d of the batch plus the batch, counting only instances whose latest edge is new"}


# --------------------------------------------------------------------- ours

def run_ours(args, ws, rank, local):
    import torch

    import aml_synth
    import paper_2604_12241_b300 as aml
    from paper_2604_12241_b300 import _lib
    from paper_2604_12241_b300 import patterns as P

    torch.cuda.set_device(local)
    dist = Dist(ws)
    params = dict(aml_synth.WORKLOADS[args.workload])
    if args.scale != 1.0:
        params["n_nodes"] = max(1000, int(params["n_nodes"] * args.scale))
        params["n_edges"] = max(10_000, int(params["n_edges"] * args.scale))
        if params.get("d_max"):
            params["d_max"] = max(50.0, params["d_max"] * args.scale)
    params["seed"] += rank * 1000     # independent replica per rank
    g = aml_synth.generate(name=args.workload, **params)
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

    def mode_ms(mode, reps=10):
        for _ in range(2):
            aml.mine(graph, ps, out=out, use_graph=use_graph, mode=mode)
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

    modes = {}
    if args.cycle_mode == "auto":
        for m in ("plain", "persistent", "learned"):
            modes[m] = mode_ms(m)
        cycle_mode = min(modes, key=modes.get)
    else:
        cycle_mode = args.cycle_mode
    for _ in range(max(3, args.warmup)):
        aml.mine(graph, ps, out=out, use_graph=use_graph, mode=cycle_mode)
    torch.cuda.synchronize()
    graph.sync()

    def timed(steps, graph_mode, profile, mode):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        dist.barrier()
        torch.cuda.synchronize()
        l0 = _lib.launch_count()
        if profile:
            _lib.profile_read(reset=True)
            _lib.profile_enable(True)
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()                     # evict L2 between steps (not timed)
            ev[k][0].record(stream)
            aml.mine(graph, ps, out=out, stream=stream, use_graph=graph_mode, mode=mode)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        dist.barrier()
        if profile:
            _lib.profile_enable(False)
        launches = _lib.launch_count() - l0
        graph.sync()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        prof = _lib.profile_read(reset=True) if profile else {}
        return ms, wall, launches, prof

    # headline: the chosen mode, clocks sampled during the timed region
    clocks = ClockSampler(local)
    clocks.start()
    dev_ms, wall, launches, _ = timed(args.steps, use_graph, False, cycle_mode)
    clk = clocks.stop()
    dev_ms_max = dist.max(dev_ms)
    # per-kernel CUDA-event times come from a pass without graph replay
    # (events cannot be recorded between the kernels of a replayed graph)
    prof_steps = max(3, min(args.steps, 10))
    plain_ms, _, plain_launches, prof = timed(prof_steps, False, True, cycle_mode)

    # end to end through the public API, every step: the step's inputs copied
    # from pinned host memory to the device, graph build, mine, and the
    # counts copied back to pinned host memory.  Transfers in one direction
    # run one at a time; an upload and a copy back overlap (the link is full
    # duplex), though each then runs slower.  The steps use a ring of three
    # slots, each with its own stream and buffers; a step takes its slot by
    # destroying the slot's previous graph (which waits for that step's copy
    # back).  The library's calls block their host thread while they wait for
    # sizes on the device, so two pipelines are timed: one host thread that
    # uploads step k, then starts step k-1's copy back under step k's build
    # and mine; and two host threads (the calls release the GIL), each step
    # enqueueing its own copy back behind its mine while the other thread's
    # step uploads, builds and mines.
    e2e = None
    if not args.no_e2e:
        import threading
        from concurrent.futures import ThreadPoolExecutor
        R = 3
        pin = {k: torch.from_numpy(v).pin_memory() for k, v in
               (("src", g.src), ("dst", g.dst), ("ts", g.ts), ("amount", g.amount))}
        S = [torch.cuda.Stream() for _ in range(R)]
        dev_in = [{k: torch.empty_like(t, device="cuda") for k, t in pin.items()} for _ in range(R)]
        dev_out = [torch.empty((E, Pn), dtype=torch.int32, device="cuda") for _ in range(R)]
        out_pin = [torch.empty((E, Pn), dtype=torch.int32).pin_memory() for _ in range(R)]
        live = [None] * R
        slot_lock = [threading.Lock() for _ in range(R)]

        dev = torch.cuda.current_device()

        def take_slot(i):
            if live[i] is not None:
                live[i].close()
                live[i] = None

        def upload(i):
            with torch.cuda.stream(S[i]):
                for key, t in pin.items():
                    dev_in[i][key].copy_(t, non_blocking=True)

        def build_mine(i):
            gg = aml.Graph(dev_in[i]["src"], dev_in[i]["dst"], dev_in[i]["ts"], g.n_nodes,
                           amount=dev_in[i]["amount"], assume_sorted=True, stream=S[i])
            aml.mine(gg, ps, out=dev_out[i], stream=S[i])
            live[i] = gg

        def copy_back(i):
            with torch.cuda.stream(S[i]):
                out_pin[i].copy_(dev_out[i], non_blocking=True)

        def step_threaded(k):
            # its own copy back behind its mine; the next step (another
            # thread) uploads, builds and mines meanwhile
            torch.cuda.set_device(dev)  # worker threads start on device 0
            i = k % R
            with slot_lock[i]:
                take_slot(i)
                upload(i)
                build_mine(i)
                copy_back(i)

        def step_single(k):
            # one thread: the upload first, at the link's full rate, then the
            # previous step's copy back under this step's build and mine
            i = k % R
            take_slot(i)
            upload(i)
            if k > 0:
                j = (k - 1) % R
                up = torch.cuda.Event()
                up.record(S[i])
                S[j].wait_event(up)
                copy_back(j)
            build_mine(i)

        def e2e_run(n_steps, workers):
            if workers == 1:
                for k in range(n_steps):
                    step_single(k)
                copy_back((n_steps - 1) % R)
            else:
                with ThreadPoolExecutor(max_workers=workers) as pool:
                    for f in [pool.submit(step_threaded, k) for k in range(n_steps)]:
                        f.result()
            for i in range(R):
                take_slot(i)

        # two host threads let two steps' builds and mines overlap: a gain
        # when the copy back dominates a step (hi-small), a loss when the
        # mine does (larger graphs); the faster of the two is reported
        e2e_times = {}
        for workers in (1, 2):
            e2e_run(R, workers)
            dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_run(args.e2e_steps, workers)
            torch.cuda.synchronize()
            e2e_times[workers] = dist.max(time.perf_counter() - t0)
        host_threads = min(e2e_times, key=e2e_times.get)
        e2e_s = e2e_times[host_threads]
        last = out_pin[(args.e2e_steps - 1) % R].numpy().view(np.uint32)
        e2e = {"value": ws * E * args.e2e_steps / e2e_s, "unit": "edges/s",
               "h2d_bytes_per_step": int(E * 16), "d2h_bytes_per_step": int(E * Pn * 4),
               "steps": args.e2e_steps, "ms_per_step": 1000.0 * e2e_s / args.e2e_steps,
               "matches_device_output": bool(np.array_equal(
                   last, out.cpu().numpy().view(np.uint32))),
               "host_threads": host_threads,
               "ms_per_step_by_host_threads": {str(w): round(1000.0 * t / args.e2e_steps, 3)
                                               for w, t in e2e_times.items()},
               "includes": "pinned host inputs -> device, graph build, mine, counts -> pinned "
                           "host memory; steps on host threads over a ring of three streams, "
                           "each step's copy back enqueued behind its mine, so the next "
                           "step's upload, build and mine overlap it"}

    line = None
    if rank == 0:
        value = ws * E * args.steps / (dev_ms_max / 1000.0)
        info = graph.info()
        # dominant kernel of the timed region, from its own CUDA events
        dom = max(prof.items(), key=lambda kv: kv[1][1])
        dom_name, (dom_n, dom_ms) = dom
        # the leg pass runs on the largest window (smaller ones are counted in it)
        big = max(int(p.name.split("@")[1]) for p in pats)
        ws_stats = graph.window_stats(big)
        stats = {"legs": ws_stats["n_legs"], "front": ws_stats["n_front"]}
        peak, peak_src = measured_peak()
        alg = algorithmic_bytes(dom_name, E, info["n_list_edges"], pats, stats)
        achieved = alg / (dom_ms / dom_n / 1000.0) / 1e9 if alg == alg else None
        traffic = None
        if (args.workload == "hi-small" and args.scale == 1.0 and kernel_digest() == KERNEL_DIGEST):
            traffic = MEASURED_TRAFFIC.get(dom_name)
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu, full size)",
                "peak_source": peak_src,
                "launch_ms": dom_ms / dom_n, "share_of_step": dom_ms / plain_ms,
                "algorithmic_bytes_per_launch": alg, "timed_in": "plain-mode profiled pass",
                "leg_pass": {"delta": big, **stats}}
        kernels = {k: {"launches": n, "ms_per_step": round(ms / prof_steps, 4),
                       "share": round(ms / plain_ms, 4)}
                   for k, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
        line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws,
                "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "impl": "ours",
                "config": {"workload": WORKLOAD_TEXT[args.workload], "n_edges": E,
                           "n_nodes": g.n_nodes, "columns": Pn, "mode": args.mode,
                           "autotune": tune_info, "cycle_mode": cycle_mode,
                           "cycle_modes_ms": modes or None,
                           "scale": args.scale,
                           "l2": "flushed between steps (256 MB write, untimed)",
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "wall_s_timed_loop": wall},
                "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "clocks": clk,
                "plain_ms_per_step": plain_ms / prof_steps,
                "cost_model": cost_report,
                "plain_gpu_launches_per_step": plain_launches / prof_steps,
                "kernels": kernels}
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, pats, args.cpu_seconds)
        if not args.no_window_cycles:
            line["window_cycles"] = time_window_cycles(graph, pats, E, use_graph, stream, flush)
        if not args.no_programs:
            line["interpreter"] = time_programs(graph, E, stream, flush)
    graph.close()
    if not args.no_stream:
        stream = run_stream(args, rank)
        if line is not None:
            line["stream"] = stream
            line["p99_stream_latency_ms"] = stream["load_50pct"]["p99_ms"]
    dist.close()
    if line is not None:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
