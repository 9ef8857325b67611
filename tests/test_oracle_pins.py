"""Pins for the CPU oracle against facts that do not come from the oracle.

* brute force over raw edge subsets (tests/brute.py) on tiny random graphs
  with timestamp ties, self-loops and several windows;
* the fuzzy SG count equals the sum of its exact temporal variants, and the
  number of admissible variants matches Sec. 4's 6! = 720 orders for a
  3-intermediary scatter-gather (tests/golden/sg_orders.txt);
* a static k-cycle under all k! timestamp permutations is a temporal cycle
  for exactly k of them, and a window cycle (any time order, Sec. 4's
  anticipatory edges) for all of them while its span fits the window;
* a window cycle count is never below the ordered one, and equal for k = 2;
* planted motifs on reserved accounts have closed-form counts;
* invariants (k | sum CYC_k, 4 | sum SG, FAN <= DEG, ...);
* DEG and FAN recomputed with numpy searchsorted / unique.
"""
import itertools
import os

import numpy as np
import pytest

import aml_synth
import oracle
from brute import admissible_orders, brute_counts, exact_sg_motif_counts

DAY = 86400
WEEK = 7 * DAY
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

ALL_SMALL = [("deg_out", 5), ("deg_in", 5), ("fan_out", 5), ("fan_in", 5),
             ("deg_out", 0), ("fan_in", 2), ("gs", 5), ("gs", 0), ("sg", 6), ("sg", 100),
             ("cyc", 2, 6), ("cyc", 3, 6), ("cyc", 4, 8), ("cyc", 5, 9), ("cyc", 3, 1000),
             ("cycw", 3, 6), ("cycw", 4, 8), ("cycw", 5, 9), ("cycw", 3, 1000)]


def _cols_10(delta):
    return [("deg_out", delta), ("deg_in", delta), ("fan_out", delta), ("fan_in", delta),
            ("gs", delta), ("sg", delta), ("cyc", 2, delta), ("cyc", 3, delta),
            ("cyc", 4, delta), ("cyc", 5, delta)]


@pytest.mark.parametrize("block", range(6))
def test_oracle_matches_brute_force(block):
    for seed in range(block * 40, block * 40 + 40):
        n = 3 + seed % 6
        E = 8 + seed % 15
        g = aml_synth.tiny_random(n, E, 10 + seed % 7, seed, self_loops=(seed % 3 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
        want = brute_counts(g.src, g.dst, g.ts, ALL_SMALL)
        got_all = og.count_all(ALL_SMALL, threads=2)
        got_ec = og.count_edges(ALL_SMALL, np.arange(E), threads=2)
        np.testing.assert_array_equal(got_all, want, err_msg=f"canonical, seed {seed}")
        np.testing.assert_array_equal(got_ec, want, err_msg=f"edge-centric, seed {seed}")


def test_brute_force_sees_every_pattern():
    """The random tiny graphs above do contain every pattern (non-vacuous)."""
    seen = np.zeros(len(ALL_SMALL), dtype=bool)
    for seed in range(240):
        n = 3 + seed % 6
        g = aml_synth.tiny_random(n, 8 + seed % 15, 10 + seed % 7, seed,
                                  self_loops=(seed % 3 == 0))
        got = oracle.OracleGraph(g.src, g.dst, g.ts, n).count_all(ALL_SMALL)
        seen |= (got > 0).any(axis=0)
    assert seen.all(), [c for c, s in zip(ALL_SMALL, seen) if not s]


def test_sg_order_counts_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sg_orders.txt"))
            if l.strip() and not l.startswith("#")]
    for k, total, ok in rows:
        assert admissible_orders(int(k)) == (int(total), int(ok))


@pytest.mark.parametrize("seed", range(12))
def test_sg_equals_sum_of_exact_variants(seed):
    rng = np.random.default_rng(1000 + seed)
    n, E = 5 + seed % 3, 14 + seed % 5
    src = rng.integers(0, n, E).astype(np.int32)
    dst = rng.integers(0, n, E).astype(np.int32)
    bad = src == dst
    dst[bad] = (dst[bad] + 1) % n
    ts = rng.permutation(40)[:E].astype(np.int32)       # distinct timestamps
    for delta in (6, 15, 100):
        total, n_variants = exact_sg_motif_counts(src, dst, ts, delta)
        assert n_variants == 6
        got = oracle.OracleGraph(src, dst, ts, n).count_all([("sg", delta)])[:, 0]
        np.testing.assert_array_equal(got.astype(np.int64), total)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_static_cycle_under_all_time_permutations(k):
    """Exactly k of the k! timestamp assignments make a temporal cycle."""
    src = np.arange(k, dtype=np.int32)
    dst = ((np.arange(k) + 1) % k).astype(np.int32)
    cols = [("cyc", j, 1000) for j in range(2, 6)]
    hits = 0
    for perm in itertools.permutations(range(k)):
        ts = np.asarray(perm, dtype=np.int32) * 10
        got = oracle.OracleGraph(src, dst, ts, k).count_all(cols)
        mine = got[:, k - 2]
        assert set(mine.tolist()) <= {0, 1} and len(set(mine.tolist())) == 1
        others = np.delete(got, k - 2, axis=1)
        assert not others.any()
        hits += int(mine[0])
        # the window excludes it once the span exceeds delta
        tight = oracle.OracleGraph(src, dst, ts, k).count_all([("cyc", k, 10 * (k - 1) - 1)])
        assert not tight.any()
    assert hits == k


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_static_window_cycle_under_all_time_permutations(k):
    """A window cycle ignores the order of its edges: every one of the k!
    timestamp assignments counts once on each edge, until the span exceeds
    the window."""
    src = np.arange(k, dtype=np.int32)
    dst = ((np.arange(k) + 1) % k).astype(np.int32)
    for perm in itertools.permutations(range(k)):
        ts = np.asarray(perm, dtype=np.int32) * 10
        og = oracle.OracleGraph(src, dst, ts, k)
        got = og.count_all([("cycw", j, 1000) for j in range(2, 6)])
        assert (got[:, k - 2] == 1).all()
        assert not np.delete(got, k - 2, axis=1).any()
        assert not og.count_all([("cycw", k, 10 * (k - 1) - 1)]).any()


def test_window_cycles_bound_ordered_cycles():
    for seed in range(60):
        g = aml_synth.tiny_random(4 + seed % 5, 30 + seed % 20, 12, 500 + seed)
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
        for d in (0, 5, 100):
            got = og.count_all([("cyc", 2, d), ("cycw", 2, d)] +
                               [(kind, k, d) for k in (3, 4, 5) for kind in ("cyc", "cycw")])
            assert (got[:, 0] == got[:, 1]).all()
            assert (got[:, 3::2] >= got[:, 2::2]).all()


def test_boundaries_and_ties():
    # two legs exactly delta apart: the span bound is inclusive
    src = np.array([0, 1, 0, 2], np.int32)
    dst = np.array([1, 3, 2, 3], np.int32)
    ts = np.array([0, 5, 5, 10], np.int32)
    og = oracle.OracleGraph(src, dst, ts, 4)
    assert og.count_all([("sg", 10)])[:, 0].tolist() == [1, 1, 1, 1]
    assert og.count_all([("sg", 9)])[:, 0].tolist() == [0, 0, 0, 0]
    # all-equal timestamps: edge ids break ties, so a leg needs a < b by id
    ts = np.zeros(4, np.int32)
    og = oracle.OracleGraph(src, dst, ts, 4)
    assert og.count_all([("sg", 0)])[:, 0].tolist() == [1, 1, 1, 1]
    og2 = oracle.OracleGraph(src[[1, 0, 3, 2]], dst[[1, 0, 3, 2]], ts, 4)
    assert og2.count_all([("sg", 0)])[:, 0].tolist() == [0, 0, 0, 0]
    # trailing window includes f with t_f == t_e - delta and ties before e
    src = np.array([0, 0, 0, 0], np.int32)
    dst = np.array([1, 2, 1, 3], np.int32)
    ts = np.array([0, 3, 3, 5], np.int32)
    got = oracle.OracleGraph(src, dst, ts, 4).count_all([("deg_out", 5), ("fan_out", 5),
                                                        ("deg_out", 2), ("fan_out", 2)])
    assert got.tolist() == [[1, 1, 1, 1], [2, 2, 1, 1], [3, 2, 2, 2], [4, 3, 3, 3]]


def test_self_loops_are_ignored():
    src = np.array([0, 1, 1, 2], np.int32)
    dst = np.array([1, 1, 2, 0], np.int32)
    ts = np.array([0, 1, 2, 3], np.int32)
    got = oracle.OracleGraph(src, dst, ts, 3).count_all(_cols_10(100))
    assert not got[1].any()
    assert got[[0, 2, 3], 7].tolist() == [1, 1, 1]     # the 3-cycle 0->1->2->0


def test_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.OracleGraph(np.array([0, 5], np.int32), np.array([1, 0], np.int32),
                           np.array([0, 1], np.int32), 3)


@pytest.fixture(scope="module")
def tiny10k():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    cols = _cols_10(DAY) + _cols_10(WEEK) + [("cycw", k, DAY) for k in (3, 4, 5)]
    return g, og, cols, og.count_all(cols)


def test_planted_motifs_have_closed_form_counts(tiny10k):
    g, og, cols, got = tiny10k
    ci = {c: i for i, c in enumerate(cols)}
    n_fresh = 0
    for m in g.motifs:
        rows = got[m.edges]
        if m.kind == "sg":
            sg = rows[:, ci[("sg", DAY)]]
            gs = rows[:, ci[("gs", DAY)]]
            if m.fresh:
                assert (sg == m.k - 1).all() and (gs == 1).all()
                n_fresh += 1
            else:
                assert (sg >= m.k - 1).all()
        else:
            cyc = rows[:, ci[("cyc", m.k, DAY)]]
            if m.fresh:
                assert (cyc == 1).all()
                for j in range(2, 6):
                    if j != m.k:
                        assert (rows[:, ci[("cyc", j, DAY)]] == 0).all()
                gs = rows[:, ci[("gs", DAY)]]
                assert gs.tolist() == [1] + [2] * (m.k - 2) + [1]
                n_fresh += 1
            else:
                assert (cyc >= 1).all()
    assert n_fresh == 50


def test_invariants(tiny10k):
    g, og, cols, got = tiny10k
    got = got.astype(np.int64)
    for d in (DAY, WEEK):
        c = {col: i for i, col in enumerate(cols)}
        for k in range(2, 6):
            assert got[:, c[("cyc", k, d)]].sum() % k == 0
        assert got[:, c[("sg", d)]].sum() % 4 == 0
        assert got[:, c[("gs", d)]].sum() % 2 == 0
        assert (got[:, c[("fan_out", d)]] <= got[:, c[("deg_out", d)]]).all()
        assert (got[:, c[("fan_in", d)]] <= got[:, c[("deg_in", d)]]).all()
        assert (got[:, c[("fan_out", d)]] >= 1).all()
        if d == DAY:
            for k in (3, 4, 5):
                assert got[:, c[("cycw", k, d)]].sum() % k == 0
                assert (got[:, c[("cycw", k, d)]] >= got[:, c[("cyc", k, d)]]).all()
    # a wider window never lowers a count
    assert (got[:, 10:20] >= got[:, :10]).all()


def test_deg_fan_against_numpy(tiny10k):
    g, og, cols, got = tiny10k
    E = g.n_edges
    ids = np.arange(E)
    for d, off in ((DAY, 0), (WEEK, 10)):
        for j, (key, other) in enumerate(((g.src, g.dst), (g.dst, g.src))):
            order = np.lexsort((ids, g.ts, key))
            comp = key[order].astype(np.int64) * 2**33 + g.ts[order]
            pos = np.empty(E, np.int64)
            pos[order] = ids
            lb = np.searchsorted(comp, key.astype(np.int64) * 2**33 + g.ts - d, side="left")
            deg = pos - lb + 1
            np.testing.assert_array_equal(got[:, off + j], deg)
            sample = np.random.default_rng(7).choice(E, 300, replace=False)
            fan = [len(np.unique(other[order[lb[e]:pos[e] + 1]])) for e in sample]
            np.testing.assert_array_equal(got[sample, off + 2 + j], fan)


def test_oracle_modes_agree_on_tiny10k(tiny10k):
    g, og, cols, got = tiny10k
    ec = og.count_edges(cols, np.arange(g.n_edges))
    np.testing.assert_array_equal(ec, got)
