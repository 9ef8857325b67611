"""Brute-force column counts straight from the definitions (tiny graphs only).

Independent of both the C oracle and the CUDA library: every instance is
found by enumerating raw edge subsets, never through adjacency lists or
windows.  Used to pin the oracle.
"""
from __future__ import annotations

import itertools
from typing import Sequence, Tuple

import numpy as np


def _prec(ts, f, e):
    return (int(ts[f]), f) < (int(ts[e]), e)


def brute_counts(src, dst, ts, cols: Sequence[Tuple]) -> np.ndarray:
    src = [int(x) for x in src]
    dst = [int(x) for x in dst]
    ts = [int(x) for x in ts]
    E = len(src)
    valid = [i for i in range(E) if src[i] != dst[i]]
    out = np.zeros((E, len(cols)), dtype=np.uint64)
    for c, col in enumerate(cols):
        kind = col[0]
        if kind in ("cyc", "cycw"):
            k, delta = int(col[1]), int(col[2])
        else:
            delta = int(col[1])
        if kind in ("deg_out", "deg_in", "fan_out", "fan_in"):
            for e in valid:
                if kind.endswith("out"):
                    win = [f for f in valid if src[f] == src[e] and not _prec(ts, e, f)
                           and ts[f] >= ts[e] - delta]
                    nb = {dst[f] for f in win}
                else:
                    win = [f for f in valid if dst[f] == dst[e] and not _prec(ts, e, f)
                           and ts[f] >= ts[e] - delta]
                    nb = {src[f] for f in win}
                out[e, c] = len(nb) if kind.startswith("fan") else len(win)
        elif kind == "gs":
            for a in valid:
                for b in valid:
                    if (dst[a] == src[b] and src[a] != dst[b] and _prec(ts, a, b)
                            and ts[b] - ts[a] <= delta):
                        out[a, c] += 1
                        out[b, c] += 1
        elif kind == "sg":
            for quad in itertools.combinations(valid, 4):
                n_assign = 0
                for a1, b1, a2, b2 in itertools.permutations(quad):
                    s, m1, m2, d = src[a1], dst[a1], dst[a2], dst[b1]
                    if not (src[a2] == s and src[b1] == m1 and src[b2] == m2 and dst[b2] == d):
                        continue
                    if len({s, m1, m2, d}) != 4:
                        continue
                    if not (_prec(ts, a1, b1) and _prec(ts, a2, b2)):
                        continue
                    tt = [ts[a1], ts[b1], ts[a2], ts[b2]]
                    if max(tt) - min(tt) > delta:
                        continue
                    n_assign += 1
                # (leg1, leg2) and (leg2, leg1) are the same unordered pair
                assert n_assign % 2 == 0
                for e in quad:
                    out[e, c] += n_assign // 2
        elif kind == "cyc":
            for sub in itertools.combinations(valid, k):
                seq = sorted(sub, key=lambda f: (ts[f], f))   # the only admissible order
                ok = all(dst[seq[i]] == src[seq[(i + 1) % k]] for i in range(k))
                ok = ok and len({src[f] for f in seq}) == k
                ok = ok and ts[seq[-1]] - ts[seq[0]] <= delta
                if ok:
                    for e in sub:
                        out[e, c] += 1
        elif kind == "cycw":
            # any k edges that chain into one simple directed cycle (distinct
            # sources, each edge's head the source of another, one orbit),
            # whatever their time order, spanning at most delta
            for sub in itertools.combinations(valid, k):
                by_src = {src[f]: f for f in sub}
                if len(by_src) != k:
                    continue
                cur, seen = sub[0], 0
                for _ in range(k):
                    if dst[cur] not in by_src:
                        break
                    cur = by_src[dst[cur]]
                    seen += 1
                orbit = {sub[0]}
                f = sub[0]
                for _ in range(k - 1):
                    if dst[f] not in by_src:
                        break
                    f = by_src[dst[f]]
                    orbit.add(f)
                ok = seen == k and cur == sub[0] and len(orbit) == k
                ok = ok and max(ts[f] for f in sub) - min(ts[f] for f in sub) <= delta
                if ok:
                    for e in sub:
                        out[e, c] += 1
        else:
            raise ValueError(kind)
    return np.minimum(out, np.uint64(0xFFFFFFFF)).astype(np.uint32)


def exact_sg_motif_counts(src, dst, ts, delta) -> np.ndarray:
    """SG counted as the sum of its exact temporal variants.

    Each exact variant fixes the full time order of the 4 edges (a1,b1,a2,b2)
    (strictly increasing timestamps; ties are not allowed here).  The
    admissible variants are the orders in which every leg's scatter precedes
    its gather: 4!/2^2 = 6 of the 24.  A conventional exact temporal-motif
    miner runs once per variant; the per-edge sum over variants must equal the
    fuzzy SG count.  Returns (per-edge sum, number of admissible variants).
    """
    src = [int(x) for x in src]
    dst = [int(x) for x in dst]
    ts = [int(x) for x in ts]
    E = len(src)
    assert len(set(ts)) == len(ts), "exact variants need distinct timestamps"
    roles = ("a1", "b1", "a2", "b2")
    variants = []
    for order in itertools.permutations(roles):
        pos = {r: i for i, r in enumerate(order)}
        if pos["a1"] < pos["b1"] and pos["a2"] < pos["b2"]:
            variants.append(order)
    # a variant and its leg-swapped twin describe the same unordered pair; keep
    # one representative per unordered pair by requiring a1's edge id < a2's
    total = np.zeros(E, dtype=np.int64)
    valid = [i for i in range(E) if src[i] != dst[i]]
    for order in variants:
        # exact motif: edges e[order[0]] < e[order[1]] < ... in time
        for a1, b1, a2, b2 in itertools.permutations(valid, 4):
            if a1 > a2:
                continue
            s, m1, m2, d = src[a1], dst[a1], dst[a2], dst[b1]
            if not (src[a2] == s and src[b1] == m1 and src[b2] == m2 and dst[b2] == d):
                continue
            if len({s, m1, m2, d}) != 4:
                continue
            e = dict(a1=a1, b1=b1, a2=a2, b2=b2)
            tt = [ts[e[r]] for r in order]
            if not all(tt[i] < tt[i + 1] for i in range(3)):
                continue
            if tt[-1] - tt[0] > delta:
                continue
            for x in (a1, b1, a2, b2):
                total[x] += 1
    return total, len(variants)


def admissible_orders(k: int) -> Tuple[int, int]:
    """(all orders, leg-respecting orders) of the 2k edges of a k-leg SG.

    Counts orderings of the edges a_1..a_k, b_1..b_k in which every a_i comes
    before its b_i, by explicit enumeration.
    """
    edges = [("a", i) for i in range(k)] + [("b", i) for i in range(k)]
    total = ok = 0
    for order in itertools.permutations(edges):
        total += 1
        pos = {x: i for i, x in enumerate(order)}
        if all(pos[("a", i)] < pos[("b", i)] for i in range(k)):
            ok += 1
    return total, ok


def _amount_rule(st):
    """(flags, lo, hi, rlo, rhi) of a stage tuple, bounds as the float32 values
    the library stores (compared in double precision)."""
    st = tuple(st) + (0, 0.0, 0.0, 0.0, 0.0)[len(st) - 9:] if len(st) < 14 else tuple(st)
    f32 = lambda v: float(np.float32(v))
    return int(st[9]), f32(st[10]), f32(st[11]), f32(st[12]), f32(st[13])


def brute_program(src, dst, ts, stages, aggregate: int, delta: int, amount=None) -> np.ndarray:
    """A stage program's counts by enumerating every tuple of edges for the
    program's edge slots (one per FOR_ALL stage, two per INTERSECT stage) and
    testing the definition on each; no neighbour lists.  aggregate 3 (SETS)
    credits each distinct edge set of the instances once.  uint64 [E]."""
    src = [int(x) for x in src]
    dst = [int(x) for x in dst]
    ts = [int(x) for x in ts]
    E = len(src)
    amt = ([float(np.float32(x)) for x in amount] if amount is not None else [0.0] * E)
    valid = [i for i in range(E) if src[i] != dst[i]]
    out = np.zeros(E, dtype=np.uint64)
    body = [tuple(int(v) for v in st[:9]) for st in stages[1:]]
    rules = [_amount_rule(st) for st in stages]
    width = sum(1 if st[0] == 1 else 2 for st in body)

    def amount_ok(rule, g, p):
        flags, lo, hi, rlo, rhi = rule
        if flags & 1 and not (lo <= amt[g] <= hi):
            return False
        if flags & 2 and not (rlo * amt[p] <= amt[g] <= rhi * amt[p]):
            return False
        return True

    def far(f, u, d):  # the other end of f if f is in u's d-list (0 out, 1 in)
        if d == 0:
            return dst[f] if src[f] == u else None
        return src[f] if dst[f] == u else None

    def before(f, e):
        return _prec(ts, f, e)

    sets = set()  # SETS: the distinct edge sets of the instances
    for e0 in valid:
        if not amount_ok(rules[0], e0, e0):  # the trigger's range (no ratio on it)
            continue
        n_bind, lasts = 0, set()
        for tup in itertools.product(valid, repeat=width):
            node = {0: src[e0], 1: dst[e0]}
            reach = {0: e0, 1: e0}
            edges, span = [e0], [e0]
            x_last, i, ok = dst[e0], 0, True
            for si, (op, a, ad, b, bd, outv, order, window, skip) in enumerate(body, 1):
                if op == 1:
                    f = tup[i]
                    i += 1
                    x = far(f, node[a], ad)
                    mine, rch = [f], f
                    if x is None or not amount_ok(rules[si], f, reach[a]):
                        ok = False
                    elif order == 1:
                        ok = before(reach[a], f)
                    elif order == 2:
                        ok = before(f, reach[a])
                    elif order == 4:
                        ok = before(e0, f)
                else:
                    fa, fb = tup[i], tup[i + 1]
                    i += 2
                    x, y = far(fa, node[a], ad), far(fb, node[b], bd)
                    mine, rch = [fa, fb], fb
                    if x is None or y is None or x != y:
                        ok = False
                    elif not (amount_ok(rules[si], fa, reach[a]) and
                              amount_ok(rules[si], fb, fa)):
                        ok = False
                    elif order == 1:
                        ok = before(reach[a], fa) and before(fa, fb)
                    elif order == 2:
                        ok = before(fb, fa) and before(fa, reach[a])
                    elif order == 3:
                        ok = before(fa, fb)
                    elif order == 4:
                        ok = before(e0, fa) and before(e0, fb)
                if not ok:
                    break
                if any((skip >> v) & 1 and node[v] == x for v in node):
                    ok = False
                    break
                if outv in node:
                    if node[outv] != x:
                        ok = False
                        break
                else:
                    node[outv], reach[outv] = x, rch
                if window == 0:
                    if not all(ts[g] >= ts[e0] - delta and (g == e0 or before(g, e0))
                               for g in mine):
                        ok = False
                        break
                else:
                    span += mine
                edges += mine
                x_last = x
            if not ok:
                continue
            if max(ts[g] for g in span) - min(ts[g] for g in span) > delta:
                continue
            if aggregate == 0:
                n_bind += 1
            elif aggregate == 1:
                lasts.add(x_last)
            elif len(set(edges)) == len(edges):
                if aggregate == 3:
                    sets.add(frozenset(edges))
                else:
                    for g in edges:
                        out[g] += 1
        if aggregate == 0:
            out[e0] = n_bind
        elif aggregate == 1:
            out[e0] = len(lasts)
    for inst in sets:
        for g in inst:
            out[g] += 1
    return out
