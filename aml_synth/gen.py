"""Synthetic temporal transaction graphs (inputs only; no counting logic).

The paper evaluates on the IBM AML datasets (Table 1: LI/HI Small, Medium,
Large) and on Trovares graphs; neither is available here, so seeded synthetic
graphs with the same node/edge counts stand in for them.

Recipe (one call = one graph):
  * background accounts 0..n_bg-1 get an out-weight and an in-weight from a
    rank-based Zipf law w_r ~ r^-alpha, scaled so the weights sum to the edge
    count and water-filled so no expected degree exceeds ``d_max``; the two
    weight vectors are independently permuted over the ids (Chung-Lu style
    preferential attachment);
  * each background edge draws src ~ out-weight and dst ~ (in-weight + 1)
    independently (drawn as per-account multinomial counts dealt in random
    order); self-loops are redrawn;
  * timestamps are uniform int32 seconds over ``days`` days (drawn, sorted
    and dealt in order to the randomly ordered edges: the same law);
  * amounts are lognormal(mu=6, sigma=2), float32;
  * planted motifs: scatter-gathers with 2..6 intermediaries and temporal
    cycles of length 3..5, all edges of one motif inside one 24h span with
    strictly increasing timestamps inside each leg/cycle; half of them use
    reserved fresh account ids (n_bg..n_nodes-1, touched by nothing else) and
    half reuse random background accounts;
  * the motif edges are merged into the time order, so edge ids are
    positions in time order (ties: background edges first, then motif
    edges in generation order).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

DAY = 86400


@dataclasses.dataclass
class Motif:
    kind: str              # "sg" or "cycle"
    k: int                 # intermediaries (sg) or cycle length
    fresh: bool            # True: all accounts reserved for this motif alone
    edges: np.ndarray      # int64 edge ids (final, time-sorted numbering)
    # sg: edges = [a_1..a_k, b_1..b_k] with a_i = s->m_i, b_i = m_i->d
    # cycle: edges = [e_1..e_k] in cyclic order, e_1 earliest


@dataclasses.dataclass
class Graph:
    src: np.ndarray        # int32 [E]
    dst: np.ndarray        # int32 [E]
    ts: np.ndarray         # int32 [E], non-decreasing
    amount: np.ndarray     # float32 [E]
    n_nodes: int
    motifs: List[Motif]
    name: str = ""
    params: Optional[dict] = None

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


def capped_zipf_weights(n: int, alpha: float, total: float, d_max: Optional[float],
                        rng: np.random.Generator) -> np.ndarray:
    """Rank-Zipf weights summing to ``total``, capped at ``d_max``, permuted."""
    r = np.arange(1, n + 1, dtype=np.float64)
    w = r ** (-alpha)
    w *= total / w.sum()
    if d_max is not None:
        for _ in range(100):
            over = w > d_max
            if not over.any():
                break
            excess = float((w[over] - d_max).sum())
            w[over] = d_max
            rest = ~over
            w[rest] += excess * w[rest] / w[rest].sum()
    return w[rng.permutation(n)]


def _draw(rng: np.random.Generator, cdf: np.ndarray, size: int) -> np.ndarray:
    u = rng.random(size)
    idx = np.searchsorted(cdf, u * cdf[-1], side="right")
    return np.minimum(idx, cdf.shape[0] - 1).astype(np.int32)


def generate(n_nodes: int, n_edges: int, alpha: float, d_max: Optional[float],
             days: float, seed: int, n_sg: int = 0, n_cycles: int = 0,
             motif_edge_frac: Optional[float] = None, name: str = "") -> Graph:
    """Build one seeded graph; ``n_edges`` counts background plus motif edges.

    Either give motif counts (``n_sg``, ``n_cycles``) or a fraction of edges
    that belong to planted motifs (split evenly between the two kinds).
    """
    rng = np.random.default_rng(seed)
    span = int(days * DAY)
    if motif_edge_frac is not None:
        budget = int(n_edges * motif_edge_frac)
        n_sg = max(2, budget // 2 // 8)        # mean sg motif: k=4 -> 8 edges
        n_cycles = max(2, budget // 2 // 4)    # mean cycle: 4 edges
    sg_k = rng.integers(2, 7, size=n_sg)
    cyc_k = rng.integers(3, 6, size=n_cycles)
    sg_fresh = np.arange(n_sg) % 2 == 0
    cyc_fresh = np.arange(n_cycles) % 2 == 0
    n_reserved = int(((sg_k + 2) * sg_fresh).sum() + (cyc_k * cyc_fresh).sum())
    n_bg = n_nodes - n_reserved
    if n_bg < 16:
        raise ValueError("too few accounts for the requested motifs")
    n_motif_edges = int(2 * sg_k.sum() + cyc_k.sum())
    n_bg_edges = n_edges - n_motif_edges
    if n_bg_edges < 0:
        raise ValueError("motifs need more edges than requested")

    w_out = capped_zipf_weights(n_bg, alpha, n_bg_edges, d_max, rng)
    w_in = capped_zipf_weights(n_bg, alpha, n_bg_edges, d_max, rng) + 1.0
    # iid draws src ~ w_out, dst ~ w_in: per-account counts (multinomial),
    # each column dealt in random order (a uniform shuffle of iid draws is
    # again iid); src == dst pairs are redrawn
    ids = np.arange(n_bg, dtype=np.int32)
    src = np.repeat(ids, rng.multinomial(n_bg_edges, w_out / w_out.sum()))
    rng.shuffle(src)
    dst = np.repeat(ids, rng.multinomial(n_bg_edges, w_in / w_in.sum()))
    rng.shuffle(dst)
    c_in = np.cumsum(w_in)
    bad = np.nonzero(src == dst)[0]
    while bad.size:
        dst[bad] = _draw(rng, c_in, bad.size)
        bad = bad[src[bad] == dst[bad]]
    # iid uniform times, independent of the (src, dst) pairs, which are in
    # random order: dealing the sorted times in order gives the same law
    ts = np.sort(rng.integers(0, span, size=n_bg_edges, dtype=np.int64))

    # planted motifs: (src, dst, t) lists plus bookkeeping of local indices
    m_src: List[int] = []
    m_dst: List[int] = []
    m_ts: List[int] = []
    plans = []
    next_fresh = n_bg

    def fresh_ids(k):
        nonlocal next_fresh
        ids = list(range(next_fresh, next_fresh + k))
        next_fresh += k
        return ids

    def bg_ids(k):
        return [int(x) for x in rng.choice(n_bg, size=k, replace=False)]

    for i in range(n_sg):
        k = int(sg_k[i])
        ids = fresh_ids(k + 2) if sg_fresh[i] else bg_ids(k + 2)
        s, d, mids = ids[0], ids[1], ids[2:]
        t0 = int(rng.integers(0, max(1, span - DAY)))
        # 2k distinct offsets inside 24h, randomly paired into legs; in each
        # leg the scatter edge takes the earlier time of its pair
        offs = rng.choice(DAY - 1, size=2 * k, replace=False)
        base = len(m_src)
        legs_a, legs_b = [], []
        for j in range(k):
            lo, hi = sorted((int(offs[2 * j]), int(offs[2 * j + 1])))
            legs_a.append((s, mids[j], t0 + lo))
            legs_b.append((mids[j], d, t0 + hi))
        for (a, b, t) in legs_a + legs_b:
            m_src.append(a); m_dst.append(b); m_ts.append(t)
        plans.append(("sg", k, bool(sg_fresh[i]), list(range(base, base + 2 * k))))
    for i in range(n_cycles):
        k = int(cyc_k[i])
        ids = fresh_ids(k) if cyc_fresh[i] else bg_ids(k)
        t0 = int(rng.integers(0, max(1, span - DAY)))
        offs = np.sort(rng.choice(DAY - 1, size=k, replace=False))
        base = len(m_src)
        for j in range(k):
            m_src.append(ids[j]); m_dst.append(ids[(j + 1) % k]); m_ts.append(t0 + int(offs[j]))
        plans.append(("cycle", k, bool(cyc_fresh[i]), list(range(base, base + k))))

    # merge the motif edges into the time order: after background edges of
    # equal time, among themselves in generation order
    m_src_a = np.asarray(m_src, dtype=np.int32)
    m_dst_a = np.asarray(m_dst, dtype=np.int32)
    m_ts_a = np.asarray(m_ts, dtype=np.int64)
    mo = np.argsort(m_ts_a, kind="stable")
    pos = np.searchsorted(ts, m_ts_a[mo], side="right")
    final = np.empty(mo.size, dtype=np.int64)
    final[mo] = pos + np.arange(mo.size)        # final edge id of each motif edge
    all_src = np.insert(src, pos, m_src_a[mo])
    all_dst = np.insert(dst, pos, m_dst_a[mo])
    all_ts = np.insert(ts, pos, m_ts_a[mo])
    amount = rng.lognormal(6.0, 2.0, size=all_ts.shape[0]).astype(np.float32)
    motifs = []
    for kind, k, fresh, loc in plans:
        motifs.append(Motif(kind, k, fresh, final[np.asarray(loc, dtype=np.int64)]))
    g = Graph(src=np.ascontiguousarray(all_src),
              dst=np.ascontiguousarray(all_dst),
              ts=np.ascontiguousarray(all_ts.astype(np.int32)),
              amount=amount, n_nodes=n_nodes, motifs=motifs, name=name,
              params=dict(n_nodes=n_nodes, n_edges=n_edges, alpha=alpha, d_max=d_max,
                          days=days, seed=seed, n_sg=n_sg, n_cycles=n_cycles))
    return g


# The five workloads (sizes of the IBM AML sets, Table 1).  Seeds are
# 20260000 + workload number.
WORKLOADS: Dict[str, dict] = {
    # 10K accounts, 100K transactions over 10 days, 50 SG + 50 cycles.
    "tiny-10k": dict(n_nodes=10_000, n_edges=100_000, alpha=1.2, d_max=1_000,
                     days=10, seed=20260001, n_sg=50, n_cycles=50),
    # HI-Small shape: 515,088 accounts, 5,078,345 transactions, 16 days.
    "hi-small": dict(n_nodes=515_088, n_edges=5_078_345, alpha=1.2, d_max=10_000,
                     days=16, seed=20260002, motif_edge_frac=0.001),
    # HI-Medium shape: 2,032,095 accounts, 31,898,238 transactions, heavier skew.
    "hi-medium": dict(n_nodes=2_032_095, n_edges=31_898_238, alpha=1.05, d_max=100_000,
                      days=16, seed=20260003, motif_edge_frac=0.001),
    # HI-Large shape: 2,070,980 accounts, 179,702,229 transactions over 90 days.
    "hi-large": dict(n_nodes=2_070_980, n_edges=179_702_229, alpha=1.2, d_max=100_000,
                     days=90, seed=20260004, motif_edge_frac=0.0005),
}


def workload(name: str, scale: float = 1.0) -> Graph:
    """One of the named workloads; ``scale`` < 1 shrinks nodes and edges."""
    p = dict(WORKLOADS[name])
    if scale != 1.0:
        p["n_nodes"] = max(1000, int(p["n_nodes"] * scale))
        p["n_edges"] = max(10_000, int(p["n_edges"] * scale))
        if p.get("d_max"):
            p["d_max"] = max(50.0, p["d_max"] * scale)
    return generate(name=name, **p)


def tiny_random(n_nodes: int, n_edges: int, t_range: int, seed: int,
                self_loops: bool = False) -> Graph:
    """Small uniform random multigraph for brute-force checks.

    Timestamps are drawn from a small range so ties are frequent; edges are
    NOT sorted by time (edge ids are arbitrary with respect to time).
    """
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n_nodes, size=n_edges).astype(np.int32)
    dst = rng.integers(0, n_nodes, size=n_edges).astype(np.int32)
    if not self_loops:
        bad = src == dst
        while bad.any():
            dst[bad] = rng.integers(0, n_nodes, size=int(bad.sum()))
            bad = src == dst
    ts = rng.integers(0, t_range, size=n_edges).astype(np.int32)
    amount = rng.lognormal(6.0, 2.0, size=n_edges).astype(np.float32)
    return Graph(src=src, dst=dst, ts=ts, amount=amount, n_nodes=n_nodes, motifs=[],
                 name=f"tiny-{seed}")
