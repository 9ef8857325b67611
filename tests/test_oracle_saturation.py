"""The oracle's saturation, pinned.

Every column is an exact count reported as a uint32 that saturates at
2^32-1 (no pattern count of the paper has a stated range; a count that does
not fit is clamped, never wrapped).  No graph small enough for the oracle
holds 2^32 instances on one edge, so the bound is an argument of the
oracle's enumerations: a test lowers it to a few units and the clamp is
reached on tiny graphs.  The pins check the clamped counts against the
brute force (``min(count, limit)``), against closed forms on a star whose
counts are known, and that the default bound leaves every count unchanged.
Planted mistakes in the clamp (wrapping instead of saturating, ignoring
the bound, clamping one below it) are compiled into copies of the oracle
and each is rejected.
"""
import os
import subprocess

import numpy as np
import pytest

import aml_synth
import oracle
from brute import brute_counts

SRC = os.path.join(os.path.dirname(oracle.__file__), "aml_oracle.c")

COLS = [("deg_out", 5), ("deg_in", 5), ("fan_out", 5), ("fan_in", 5), ("gs", 5), ("sg", 6),
        ("sg", 100), ("cyc", 2, 6), ("cyc", 3, 6), ("cyc", 4, 8), ("cycw", 3, 6)]

LIMITS = (1, 2, 3, 7)


def _graphs():
    # small node counts and long windows give counts well above the limits
    for seed in range(24):
        n = 3 + seed % 4
        E = 10 + seed % 9
        yield aml_synth.tiny_random(n, E, 6 + seed % 5, 9000 + seed, self_loops=(seed % 3 == 0))


def _clamp_pins_reject(lib) -> bool:
    reached = 0
    for g in _graphs():
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes, lib=lib)
        full = brute_counts(g.src, g.dst, g.ts, COLS)
        if not np.array_equal(og.count_all(COLS, threads=1), full):
            return True
        for lim in LIMITS:
            want = np.minimum(full, lim).astype(np.uint32)
            reached += int((full > lim).sum())
            if not np.array_equal(og.count_all(COLS, threads=1, limit=lim), want):
                return True
            if not np.array_equal(og.count_edges(COLS, np.arange(g.n_edges), threads=1,
                                                 limit=lim), want):
                return True
    assert reached > 100, "the pin graphs must exceed the limits often"
    return False


def _star(n_in: int, n_out: int):
    """Hub 0; senders 1..n_in send to it first, then it pays receivers
    n_in+1..n_in+n_out, one second apart: every gather edge is in n_out
    gather-scatter 2-paths and every scatter edge in n_in (all ends distinct,
    all within a day)."""
    src = np.array(list(range(1, n_in + 1)) + [0] * n_out, dtype=np.int32)
    dst = np.array([0] * n_in + list(range(n_in + 1, n_in + n_out + 1)), dtype=np.int32)
    ts = np.arange(n_in + n_out, dtype=np.int32)
    return src, dst, ts, n_in + n_out + 1


def test_clamped_counts_equal_min_of_brute_force():
    assert not _clamp_pins_reject(oracle._load())


@pytest.mark.parametrize("limit", [1, 3, 5, 8, 9, 1000])
def test_star_closed_form(limit):
    n_in, n_out = 3, 8
    src, dst, ts, n = _star(n_in, n_out)
    og = oracle.OracleGraph(src, dst, ts, n)
    cols = [("gs", 86400), ("deg_out", 86400), ("fan_in", 86400)]
    got = og.count_all(cols, limit=limit)
    gs = np.array([n_out] * n_in + [n_in] * n_out, dtype=np.int64)
    deg_out = np.array([1] * n_in + list(range(1, n_out + 1)), dtype=np.int64)
    fan_in = np.array(list(range(1, n_in + 1)) + [1] * n_out, dtype=np.int64)
    for c, exact in enumerate((gs, deg_out, fan_in)):
        np.testing.assert_array_equal(got[:, c], np.minimum(exact, limit))
    # a count exactly at the limit is kept, not lowered
    if limit == n_out:
        assert np.all(got[:n_in, 0] == n_out)
    if limit == n_in:
        assert np.all(got[n_in:, 0] == n_in)


def test_default_limit_changes_nothing():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    cols = [("deg_out", 86400), ("gs", 86400), ("sg", 86400), ("cyc", 3, 86400)]
    a = og.count_all(cols)
    b = og.count_all(cols, limit=0xFFFFFFFF)
    np.testing.assert_array_equal(a, b)
    ids = np.arange(0, g.n_edges, 997)
    np.testing.assert_array_equal(og.count_edges(cols, ids, limit=int(a.max())), a[ids])


def test_limit_zero_is_refused():
    src, dst, ts, n = _star(2, 2)
    og = oracle.OracleGraph(src, dst, ts, n)
    with pytest.raises(ValueError):
        og.count_all([("gs", 10)], limit=0)


CLAMP_MUTANTS = [
    ("clamp-wraps", "return v > (uint64_t)limit ? limit : (uint32_t)v;",
     "return (uint32_t)(v & (uint64_t)limit);"),
    ("clamp-ignores-limit", "return v > (uint64_t)limit ? limit : (uint32_t)v;",
     "return v > 0xffffffffull ? 0xffffffffu : (uint32_t)v;"),
    ("clamp-one-below", "return v > (uint64_t)limit ? limit : (uint32_t)v;",
     "return v >= (uint64_t)limit ? limit - 1 : (uint32_t)v;"),
]


@pytest.mark.parametrize("name,orig,mutated", CLAMP_MUTANTS, ids=[m[0] for m in CLAMP_MUTANTS])
def test_clamp_pins_reject_mutant(tmp_path, name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(orig, mutated))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-I", os.path.dirname(SRC), "-o", str(so), str(path)])
    lib = oracle.load_library(str(so))
    assert _clamp_pins_reject(lib), f"mutant {name} survived the saturation pins"
