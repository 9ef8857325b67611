"""Pins for the "Stack" reading (Sec. 8, Fig. 9 benchmark a Stack pattern
that the text never defines; read as the stacked bipartite: senders s1, s2
each paying both middle accounts m1, m2, which each pay both receivers
r1, r2, six distinct accounts, all eight transfers within delta).

The oracle evaluates the stage program (og_program_count, SETS aggregate);
these tests set it against a raw-edge enumeration of the definition that
uses no program semantics (every choice of the three account pairs, every
choice of one edge for each of the eight account pairs), against closed
forms on planted stacks, and check the 8 bindings per instance that the
GPU's division relies on.
"""
import dataclasses
import itertools

import numpy as np
import pytest

import oracle
from paper_2604_12241_b300 import patterns as P


def _tuples(pattern):
    return [dataclasses.astuple(s) for s in pattern.stages]


def brute_stacks(src, dst, ts, delta):
    """Per edge: the stacks whose eight edges include it, each once."""
    E = len(src)
    pairs = {}
    for e in range(E):
        if src[e] != dst[e]:
            pairs.setdefault((int(src[e]), int(dst[e])), []).append(e)
    nodes = sorted({int(x) for x in src} | {int(x) for x in dst})
    out = np.zeros(E, dtype=np.uint64)
    for s1, s2 in itertools.combinations(nodes, 2):
        rest = [n for n in nodes if n not in (s1, s2)]
        for m1, m2 in itertools.combinations(rest, 2):
            first = [pairs.get((s, m), []) for s in (s1, s2) for m in (m1, m2)]
            if not all(first):
                continue
            for r1, r2 in itertools.combinations([n for n in rest if n not in (m1, m2)], 2):
                second = [pairs.get((m, r), []) for m in (m1, m2) for r in (r1, r2)]
                if not all(second):
                    continue
                for combo in itertools.product(*first, *second):
                    t = [int(ts[e]) for e in combo]
                    if max(t) - min(t) <= delta:
                        for e in combo:
                            out[e] += 1
    return out


def _dense_graph(seed, n, E, t_max):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, E).astype(np.int32)
    dst = rng.integers(0, n, E).astype(np.int32)
    ts = np.sort(rng.integers(0, t_max, E)).astype(np.int32)
    return src, dst, ts


def test_stack_sets_match_the_raw_edge_enumeration():
    checked = 0
    for seed in range(8):
        n, E = 6 + seed % 3, 40 + 4 * seed
        src, dst, ts = _dense_graph(9100 + seed, n, E, 12)
        og = oracle.OracleGraph(src, dst, ts, n)
        for delta in (2, 5, 100):
            pat = P.stack(delta)
            want = brute_stacks(src, dst, ts, delta)
            got = og.program_count(_tuples(pat), oracle.AGG_SETS, delta, threads=2)
            np.testing.assert_array_equal(got.astype(np.uint64), want,
                                          err_msg=f"seed {seed}, delta {delta}")
            checked += int((want > 0).sum())
    assert checked > 50


def test_every_stack_is_found_by_eight_bindings():
    """Any of its four first-layer edges as the trigger, and its two
    receivers in either order: the per-binding (INSTANCES) count is exactly
    8 times the per-instance one, which the GPU divides by."""
    checked = 0
    for seed in range(5):
        src, dst, ts = _dense_graph(9200 + seed, 7, 50, 10)
        og = oracle.OracleGraph(src, dst, ts, 7)
        for delta in (3, 100):
            pat = P.stack(delta)
            per_binding = og.program_count(_tuples(pat), oracle.AGG_INSTANCES, delta, threads=2)
            want = brute_stacks(src, dst, ts, delta)
            np.testing.assert_array_equal(per_binding.astype(np.uint64), want * np.uint64(8))
            checked += int((want > 0).sum())
    assert checked > 50


def _planted(extra=()):
    # s1=0, s2=1, m1=2, m2=3, r1=4, r2=5: the first layer at t = 10..13, the
    # second at t = 20..23
    edges = [(0, 2, 10), (0, 3, 11), (1, 2, 12), (1, 3, 13),
             (2, 4, 20), (2, 5, 21), (3, 4, 22), (3, 5, 23)] + list(extra)
    edges.sort(key=lambda e: e[2])
    src = np.array([e[0] for e in edges], dtype=np.int32)
    dst = np.array([e[1] for e in edges], dtype=np.int32)
    ts = np.array([e[2] for e in edges], dtype=np.int32)
    return src, dst, ts


def test_planted_stack_closed_forms():
    src, dst, ts = _planted()
    og = oracle.OracleGraph(src, dst, ts, 6)
    # one instance: 1 on each of its eight edges, inside any window >= its 13 s span
    for delta in (13, 1000):
        got = og.program_count(_tuples(P.stack(delta)), oracle.AGG_SETS, delta)
        np.testing.assert_array_equal(got, np.ones(8, dtype=got.dtype))
    got = og.program_count(_tuples(P.stack(12)), oracle.AGG_SETS, 12)
    assert not got.any()  # the span is 13 s
    # a parallel first-layer edge s1 -> m1: two instances, which share the
    # other seven edges
    src, dst, ts = _planted([(0, 2, 15)])
    og = oracle.OracleGraph(src, dst, ts, 6)
    got = og.program_count(_tuples(P.stack(100)), oracle.AGG_SETS, 100)
    par = [i for i in range(len(src)) if (src[i], dst[i]) == (0, 2)]
    want = np.full(len(src), 2, dtype=got.dtype)
    want[par] = 1
    np.testing.assert_array_equal(got, want)
    # a third receiver paid by both middle accounts: C(3, 2) = 3 instances;
    # the first layer is in all three, each second-layer edge in two
    src, dst, ts = _planted([(2, 6, 24), (3, 6, 25)])
    og = oracle.OracleGraph(src, dst, ts, 7)
    got = og.program_count(_tuples(P.stack(100)), oracle.AGG_SETS, 100)
    first = (dst == 2) | (dst == 3)
    np.testing.assert_array_equal(got[first], 3)
    np.testing.assert_array_equal(got[~first], 2)


@pytest.mark.parametrize("drop", range(8))
def test_an_incomplete_stack_counts_nothing(drop):
    src, dst, ts = _planted()
    keep = np.arange(8) != drop
    og = oracle.OracleGraph(src[keep], dst[keep], ts[keep], 6)
    assert not og.program_count(_tuples(P.stack(100)), oracle.AGG_SETS, 100).any()


def test_stack_accounts_must_be_distinct():
    """A receiver that is also a sender (r1 = s2) makes no stack: the
    program's skips keep the six accounts distinct."""
    edges = [(0, 2, 10), (0, 3, 11), (1, 2, 12), (1, 3, 13),
             (2, 1, 20), (2, 5, 21), (3, 1, 22), (3, 5, 23)]
    src = np.array([e[0] for e in edges], dtype=np.int32)
    dst = np.array([e[1] for e in edges], dtype=np.int32)
    ts = np.array([e[2] for e in edges], dtype=np.int32)
    og = oracle.OracleGraph(src, dst, ts, 6)
    assert not og.program_count(_tuples(P.stack(100)), oracle.AGG_SETS, 100).any()
    assert not brute_stacks(src, dst, ts, 100).any()
