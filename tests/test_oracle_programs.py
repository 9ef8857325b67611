"""Pins for the oracle's generic interpretation of stage programs
(og_program_count), against facts that do not come from it:

* brute force over raw edge tuples (tests/brute.py, brute_program) for
  programs no pattern family matches, on tiny random graphs with ties and
  self-loops;
* every family's own program, interpreted generically, gives that family's
  counts from the oracle's separate family enumerations (themselves pinned
  by brute force): DEG/FAN through EDGES/DISTINCT, GS and CYC_k and CYCW_k
  through INSTANCES, and SG twice over (each pair of legs is found once from
  each scatter edge, or once from each gather edge);
* a program with contradictory constraints counts nothing;
* the n-intermediary scatter-gather programs ("at least N", Sec. 4) give
  n! * C(k - 1, n - 1) on every edge of a planted isolated k-intermediary
  scatter-gather, and 0 when k < n.
"""
import math
import dataclasses

import numpy as np
import pytest

import aml_synth
import oracle
from brute import brute_program
from paper_2604_12241_b300 import patterns as P
from programs import AMOUNT_PROGRAMS, AMOUNT_VALUES, NOVEL


def _tuples(pattern):
    return [dataclasses.astuple(s) for s in pattern.stages]


@pytest.mark.parametrize("name", sorted(NOVEL))
def test_program_oracle_matches_brute_force(name):
    stages, agg = NOVEL[name]
    width = sum(1 if s[0] == 1 else 2 for s in stages[1:])
    n_graphs = 14 if width <= 2 else 6
    for seed in range(n_graphs):
        n = 3 + seed % 5
        E = (14 if width <= 2 else 10) + seed % 5
        g = aml_synth.tiny_random(n, E, 8 + seed % 6, 1000 + seed, self_loops=(seed % 3 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
        for delta in (0, 3, 1000):
            want = brute_program(g.src, g.dst, g.ts, stages, agg, delta)
            got = og.program_count(stages, agg, delta, threads=2)
            np.testing.assert_array_equal(got, want, err_msg=f"{name}, seed {seed}, delta {delta}")


def test_contradictory_program_counts_nothing():
    stages, agg = NOVEL["empty_trailing_after"]
    g = aml_synth.tiny_random(20, 400, 50, 7)
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    assert not og.program_count(stages, agg, 10**6).any()


def _family_cases(delta):
    out = [(P.deg_out(delta), ("deg_out", delta), 1), (P.deg_in(delta), ("deg_in", delta), 1),
           (P.fan_out(delta), ("fan_out", delta), 1), (P.fan_in(delta), ("fan_in", delta), 1),
           (P.gather_scatter(delta), ("gs", delta), 1),
           (P.gather_scatter(delta, mirrored=True), ("gs", delta), 1),
           (P.scatter_gather(delta), ("sg", delta), 2),
           (P.scatter_gather(delta, trigger="gather"), ("sg", delta), 2)]
    for k in range(2, 6):
        out.append((P.cycle(k, delta), ("cyc", k, delta), 1))
        if k >= 3:
            out.append((P.cycle(k, delta, closing="intersect"), ("cyc", k, delta), 1))
            out.append((P.window_cycle(k, delta), ("cycw", k, delta), 1))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_family_programs_interpreted_generically(seed):
    g = aml_synth.tiny_random(25, 500, 400, 77 + seed, self_loops=(seed == 1))
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    for delta in (30, 150):
        cases = _family_cases(delta)
        fam = og.count_all([c[1] for c in cases], threads=4)
        for j, (pat, col, factor) in enumerate(cases):
            got = og.program_count(_tuples(pat), pat.aggregate, pat.delta, threads=4)
            np.testing.assert_array_equal(got.astype(np.uint64),
                                          fam[:, j].astype(np.uint64) * factor,
                                          err_msg=f"{pat.name} (seed {seed})")


def test_n_intermediary_scatter_gather_closed_form():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    fresh = [m for m in g.motifs if m.kind == "sg" and m.fresh]
    assert len(fresh) >= 10 and {m.k for m in fresh} >= {2, 3, 4}
    for n in (2, 3, 4):
        pat = P.scatter_gather_n(n, P.DAY)
        got = og.program_count(_tuples(pat), pat.aggregate, pat.delta)
        for m in fresh:
            want = math.factorial(n) * math.comb(m.k - 1, n - 1) if m.k >= n else 0
            assert (got[m.edges] == want).all(), (n, m.k, got[m.edges])


def test_node_level_scatter_gather_closed_form():
    """Distinct other intermediaries per scatter edge: k - 1 on the scatter
    edges of a planted isolated k-SG, 0 on its gather edges, and never more
    than the edge-level pair count of the same trigger."""
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    pat = P.scatter_gather_nodes(P.DAY)
    got = og.program_count(_tuples(pat), pat.aggregate, pat.delta)
    pairs = og.program_count(_tuples(P.scatter_gather(P.DAY)), P.AGG_EDGES, P.DAY)
    assert (got.astype(np.int64) <= pairs.astype(np.int64)).all()
    fresh = [m for m in g.motifs if m.kind == "sg" and m.fresh]
    assert fresh
    for m in fresh:
        scatter = [e for e in m.edges if g.dst[e] != g.dst[m.edges[-1]]]
        gather = [e for e in m.edges if e not in scatter]
        assert len(scatter) == len(gather) == m.k
        assert (got[scatter] == m.k - 1).all() and (got[gather] == 0).all()


def test_n_intermediary_scatter_gather_brute_force():
    """Legs s -> m -> d through four candidate intermediaries at random times
    (some out of order, one repeated), plus noise edges."""
    pat = P.scatter_gather_n(3, 0)
    n_nonzero = 0
    for seed in range(5):
        rng = np.random.default_rng(900 + seed)
        src, dst = [], []
        for m in range(2, 6):
            for _ in range(1 + (m == 2)):
                src += [0, m]
                dst += [m, 1]
        for _ in range(2):
            a, b = rng.integers(0, 6, 2)
            src.append(int(a))
            dst.append(int(b))
        ts = rng.integers(0, 8, len(src))
        og = oracle.OracleGraph(src, dst, ts, 6)
        for delta in (3, 1000):
            want = brute_program(src, dst, ts, _tuples(pat), pat.aggregate, delta)
            got = og.program_count(_tuples(pat), pat.aggregate, delta, threads=2)
            np.testing.assert_array_equal(got, want, err_msg=f"seed {seed}, delta {delta}")
            n_nonzero += int(want.any())
    assert n_nonzero >= 3


@pytest.mark.parametrize("name", sorted(AMOUNT_PROGRAMS))
def test_amount_programs_match_brute_force(name):
    """Amount constraints (RANGE on the trigger and stages, RATIO along the
    walk) against the brute force, amounts from a small set so that ratio
    bounds meet exact pairs."""
    stages, agg = AMOUNT_PROGRAMS[name]
    width = sum(1 if s[0] == 1 else 2 for s in stages[1:])
    n_nonzero = 0
    for seed in range(16):
        n = 3 + seed % 3
        E = (14 if width <= 2 else 10) + seed % 4
        g = aml_synth.tiny_random(n, E, 8 + seed % 5, 2000 + seed, self_loops=(seed % 3 == 0))
        rng = np.random.default_rng(seed)
        # plus a triangle 0 -> 1 -> 2 -> 0 and a two-leg scatter-gather
        # 0 -> {1, 2} -> 3 whose amounts fall off by 5% a hop, at random times
        src = np.concatenate([g.src, [0, 1, 2, 0, 0, 1, 2]]).astype(np.int32)
        dst = np.concatenate([g.dst, [1, 2, 0, 1, 2, 3, 3]]).astype(np.int32)
        ts = np.concatenate([g.ts, np.sort(rng.integers(0, 8, 3)),
                             np.sort(rng.integers(0, 8, 2)), np.sort(rng.integers(4, 12, 2))])
        amount = np.concatenate([rng.choice(AMOUNT_VALUES, E), [100.0, 95.0, 90.0],
                                 [100.0, 100.0], [95.0, 95.0]]).astype(np.float32)
        n = max(n, 4)
        og = oracle.OracleGraph(src, dst, ts, n, amount=amount)
        for delta in (3, 1000):
            want = brute_program(src, dst, ts, stages, agg, delta, amount=amount)
            got = og.program_count(stages, agg, delta, threads=2)
            np.testing.assert_array_equal(got, want, err_msg=f"{name}, seed {seed}, delta {delta}")
            n_nonzero += int(want.any())
    assert n_nonzero >= 2


def test_amount_constraints_only_remove():
    """A constrained program counts at most what the same program without the
    constraints counts, edge by edge; with bounds that admit every amount it
    counts the same."""
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount)
    for name, (stages, agg) in AMOUNT_PROGRAMS.items():
        free = [tuple(s[:9]) for s in stages]
        loose = [tuple(s[:9]) + ((s[9], 0.0, 3.4e38, 0.0, 3.4e38) if len(s) > 9 else ())
                 for s in stages]
        c = og.program_count(stages, agg, P.DAY).astype(np.int64)
        f = og.program_count(free, agg, P.DAY).astype(np.int64)
        l = og.program_count(loose, agg, P.DAY).astype(np.int64)
        assert (c <= f).all(), name
        np.testing.assert_array_equal(l, f, err_msg=name)


@pytest.mark.parametrize("n_in,n_out", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 2)])
def test_gather_scatter_n_closed_form(n_in, n_out):
    """A planted star, k_in senders into a hub and then k_out receivers out of
    it, every gather before every scatter: a gather edge lies in
    C(k_in-1, n_in-1) (n_in-1)! k_out!/(k_out-n_out)! bindings, a scatter
    edge in C(k_in, n_in) (n_in-1)! n_out (k_out-1)!/(k_out-n_out)!."""
    k_in, k_out, hub = 4, 3, 0
    src = [1 + i for i in range(k_in)] + [hub] * k_out
    dst = [hub] * k_in + [1 + k_in + i for i in range(k_out)]
    ts = list(range(k_in + k_out))
    og = oracle.OracleGraph(src, dst, ts, 1 + k_in + k_out)
    pat = P.gather_scatter_n(n_in, n_out, 100)
    got = og.program_count(_tuples(pat), pat.aggregate, pat.delta)
    f, c = math.factorial, math.comb
    perm = lambda n, k: f(n) // f(n - k)
    want_g = c(k_in - 1, n_in - 1) * f(n_in - 1) * perm(k_out, n_out)
    want_s = c(k_in, n_in) * f(n_in - 1) * n_out * perm(k_out - 1, n_out - 1)
    assert (got[:k_in] == want_g).all() and (got[k_in:] == want_s).all(), got
    if (n_in, n_out) == (1, 1):  # the GS program: equals the family
        np.testing.assert_array_equal(got, og.count_all([("gs", 100)])[:, 0])


def test_gather_scatter_n_brute_force():
    """A hub 0 with three senders and three receivers at random times (so
    some scatters precede some gathers), a repeated sender, and noise."""
    pat = P.gather_scatter_n(2, 2, 0)
    n_nonzero = 0
    for seed in range(6):
        rng = np.random.default_rng(5000 + seed)
        src = [1, 2, 3, 1, 0, 0, 0] + list(rng.integers(0, 7, 3))
        dst = [0, 0, 0, 0, 4, 5, 1] + list(rng.integers(0, 7, 3))
        ts = list(rng.integers(0, 8, len(src)))
        og = oracle.OracleGraph(src, dst, ts, 7)
        for delta in (3, 1000):
            want = brute_program(src, dst, ts, _tuples(pat), pat.aggregate, delta)
            got = og.program_count(_tuples(pat), pat.aggregate, delta, threads=2)
            np.testing.assert_array_equal(got, want, err_msg=f"seed {seed}, delta {delta}")
            n_nonzero += int(want.any())
    assert n_nonzero >= 3


def _brute_sg_sets(src, dst, ts, k, delta):
    """Per edge, the k-intermediary scatter-gathers it belongs to, each
    counted once as a set: k legs s -> m_i -> d (scatter before gather in
    (t, id) order, s, d and the m_i distinct) with pairwise distinct
    intermediaries and all 2k edges within delta.  Enumerated from the raw
    edge list (no neighbour lists)."""
    import itertools
    E = len(src)
    prec = lambda f, e: (int(ts[f]), f) < (int(ts[e]), e)
    legs = [(a, b) for a in range(E) for b in range(E)
            if src[a] != dst[a] and src[b] != dst[b] and dst[a] == src[b]
            and src[a] != dst[b] and prec(a, b)]
    out = np.zeros(E, dtype=np.uint64)
    by_pair = {}
    for a, b in legs:
        by_pair.setdefault((int(src[a]), int(dst[b])), []).append((a, b))
    for group in by_pair.values():
        for combo in itertools.combinations(group, k):
            mids = {int(dst[a]) for a, _ in combo}
            if len(mids) != k:
                continue
            edges = [e for leg in combo for e in leg]
            t = [int(ts[e]) for e in edges]
            if max(t) - min(t) > delta:
                continue
            for e in edges:
                out[e] += 1
    return out


@pytest.mark.parametrize("k", [2, 3])
def test_exact_size_scatter_gather_is_the_at_least_program_over_k_factorial(k):
    """Exact-size bins: the k-intermediary scatter-gathers an edge belongs
    to, each counted once (a set of k legs), equal the "at least k" program's
    count (ordered k-tuples of legs) divided by k!, on small random graphs
    with ties, parallel edges and self-loops (brute force over raw edges)."""
    pat = P.scatter_gather_n(k, 0)
    checked = 0
    for seed in range(12):
        rng = np.random.default_rng(4000 + seed)
        n, E = 5, 24 + seed % 8
        src = rng.integers(0, n, E).astype(np.int32)
        dst = rng.integers(0, n, E).astype(np.int32)
        ts = rng.integers(0, 7, E).astype(np.int32)
        og = oracle.OracleGraph(src, dst, ts, n)
        for delta in (2, 6):
            got = og.program_count(_tuples(pat), pat.aggregate, delta, threads=1)
            want = _brute_sg_sets(src, dst, ts, k, delta)
            np.testing.assert_array_equal(got.astype(np.uint64),
                                          want * np.uint64(math.factorial(k)))
            checked += int((want > 0).sum())
    assert checked > 20


# ---- the SETS aggregate: each distinct edge set of the instances once ----

_SETS_NOVEL = ("path3", "gs_any_order", "common_out", "fan_pairs", "leg_triangle", "closing_in")


def _sets_cases():
    cases = {name: NOVEL[name][0] for name in _SETS_NOVEL}
    for n in (2, 3):
        cases[f"sg{n}"] = _tuples(P.scatter_gather_n(n, 0))
    return cases


@pytest.mark.parametrize("name", sorted(_sets_cases()))
def test_sets_aggregate_matches_brute_force(name):
    """SETS credits every distinct edge set of the program's instances once,
    whichever triggers and stage orders find it (brute force over raw edge
    tuples, collecting the sets)."""
    stages = _sets_cases()[name]
    width = sum(1 if s[0] == 1 else 2 for s in stages[1:])
    for seed in range(10 if width <= 2 else 5):
        n = 3 + seed % 4
        E = (13 if width <= 2 else 10) + seed % 4
        g = aml_synth.tiny_random(n, E, 8 + seed % 6, 7000 + seed, self_loops=(seed % 3 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
        for delta in (0, 3, 1000):
            want = brute_program(g.src, g.dst, g.ts, stages, oracle.AGG_SETS, delta)
            got = og.program_count(stages, oracle.AGG_SETS, delta, threads=2)
            np.testing.assert_array_equal(got, want, err_msg=f"{name}, seed {seed}, delta {delta}")


@pytest.mark.parametrize("k", [2, 3, 4])
def test_sets_of_the_k_intermediary_program_is_the_exact_motif(k):
    """Exact-size bins as a column: the SETS aggregate of the k-intermediary
    scatter-gather program counts every set of k legs (one source, one
    destination, pairwise distinct intermediaries, each leg in order, all 2k
    edges within delta) once on each of its edges: the raw-edge brute force
    of exact k-intermediary motifs."""
    pat = P.scatter_gather_n(k, 0)
    checked = 0
    for seed in range(10):
        rng = np.random.default_rng(5000 + seed)
        n, E = (5, 24 + seed % 8) if k < 4 else (6, 48 + seed % 6)
        src = rng.integers(0, n, E).astype(np.int32)
        dst = rng.integers(0, n, E).astype(np.int32)
        ts = rng.integers(0, 7, E).astype(np.int32)
        og = oracle.OracleGraph(src, dst, ts, n)
        for delta in (2, 6):
            got = og.program_count(_tuples(pat), oracle.AGG_SETS, delta, threads=1)
            want = _brute_sg_sets(src, dst, ts, k, delta)
            np.testing.assert_array_equal(got.astype(np.uint64), want)
            checked += int((want > 0).sum())
    assert checked > 20


def test_sets_of_two_intermediaries_is_the_sg_column():
    """The 2-intermediary set is an SG instance (an unordered pair of legs):
    the SETS aggregate of that program equals the oracle's SG family
    column, which its separate enumeration computes (pinned by brute force)."""
    for seed, delta in ((1, 20), (2, 60), (3, 1000)):
        g = aml_synth.tiny_random(12, 400, 200, 8100 + seed, self_loops=(seed == 2))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
        pat = P.scatter_gather_n(2, delta)
        got = og.program_count(_tuples(pat), oracle.AGG_SETS, delta)
        want = og.count_all([("sg", delta)])[:, 0]
        assert want.sum() > 0
        np.testing.assert_array_equal(got, want)
