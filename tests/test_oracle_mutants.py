"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake (a dropped term, a flipped comparison, an
off-by-one index, a wrong operand, an ordered hop in a window cycle) in a temporary copy of the oracle's C
source, compiles it on the CPU, and checks that the brute-force pins reject
the mutant.  The oracle under oracle/ is never modified.
"""
import os
import subprocess

import numpy as np
import pytest

import aml_synth
import oracle
from brute import brute_counts, brute_program
from programs import AMOUNT_PROGRAMS, AMOUNT_VALUES, NOVEL

SRC = os.path.join(os.path.dirname(oracle.__file__), "aml_oracle.c")

# (name, original text, mutated text) -- every original must occur exactly once
MUTANTS = [
    ("prec-tie-reversed", "(g->ts[f] == g->ts[e] && f < e)", "(g->ts[f] == g->ts[e] && f > e)"),
    ("find-start-exclusive", "if ((int64_t)g->ts[list[mid]] < tmin) lo",
     "if ((int64_t)g->ts[list[mid]] <= tmin) lo"),
    ("deg-off-by-one", "return (uint64_t)(pos - lo + 1);", "return (uint64_t)(pos - lo);"),
    ("fan-counts-repeats", "if (i == 0 || buf[i] != buf[i - 1]) ++d;", "++d;"),
    ("gs-keeps-reciprocal", "      if (g->dst[b] == x) continue;                       /* skip_if: y == x */\n",
     ""),
    ("gs-window-open", "if ((int64_t)g->ts[b] - g->ts[a] > delta) break;  /* break_if",
     "if ((int64_t)g->ts[b] - g->ts[a] >= delta) break;  /* break_if"),
    ("sg-same-intermediary", "if (m2 <= m1 || m2 == d) continue;", "if (m2 < m1 || m2 == d) continue;"),
    ("sg-span-from-leg1", "int64_t lo2 = lo < g->ts[a2] ? lo : g->ts[a2];", "int64_t lo2 = lo;"),
    ("sg-leg-order-dropped",
     "for (int64_t q = first_after(g, g->out_list, g->out_start[m2], q_end, a2); q < q_end; ++q) {",
     "for (int64_t q = g->out_start[m2]; q < q_end; ++q) {"),
    ("sg-partner-wrong-operand", "if (g->src[a2] != s) continue;", "if (g->src[a2] == s) continue;"),
    ("cyc-credit-skips-first", "for (int j = 0; j < depth; ++j) add(",
     "for (int j = 1; j < depth; ++j) add("),
    ("cyc-not-simple", "for (int j = 1; j <= depth; ++j) seen |= (c->nodes[j] == x);",
     "for (int j = 2; j <= depth; ++j) seen |= (c->nodes[j] == x);"),
    ("ec-cyc-descents", "if (nd == 1 || c->window) c->cnt++;", "if (nd <= 2 || c->window) c->cnt++;"),
    ("cycw-after-previous-hop", "int64_t after = c->window ? c->edges[0] : c->edges[depth - 1];",
     "int64_t after = c->edges[depth - 1];"),
    ("ec-cycw-prunes-descents", "if (z == x || (nd > 1 && !c->window)) continue;",
     "if (z == x || nd > 1) continue;"),
]

# mistakes in the generic interpretation of stage programs, caught by the
# brute-force program pins
PROGRAM_MUTANTS = [
    ("prog-intersect-before-flipped",
     "if (s->order == OG_ORD_BEFORE && !(prec(g, fb, fa) && prec(g, fa, ra))) continue;",
     "if (s->order == OG_ORD_BEFORE && !(prec(g, fa, fb) && prec(g, fa, ra))) continue;"),
    ("prog-trailing-admits-later", "&& (f == c->e0 || prec(g, f, c->e0));", ";"),
    ("prog-instances-repeat-edges", "        if (c->edges[i] == c->edges[j]) return;\n", ""),
    ("prog-closing-ignored", "  if (s->out_var < bound && c->node[s->out_var] != x) return 0;\n", ""),
    ("prog-span-open", "if (tmax - tmin > c->delta) return;", "if (tmax - tmin >= c->delta) return;"),
    ("prog-distinct-counts-all", "if (c->seen[i] == x_last) return;", "if (0) return;"),
    ("prog-leg-reversed", "if (s->order == OG_ORD_LEG && !prec(g, fa, fb)) continue;",
     "if (s->order == OG_ORD_LEG && !prec(g, fb, fa)) continue;"),
]

COLS = [("deg_out", 5), ("deg_in", 5), ("fan_out", 5), ("fan_in", 5), ("gs", 5), ("sg", 6),
        ("sg", 100), ("cyc", 2, 6), ("cyc", 3, 6), ("cyc", 4, 8), ("cyc", 5, 9),
        ("cycw", 3, 6), ("cycw", 4, 8)]


def _pins_reject(lib) -> bool:
    for seed in range(80):
        n = 3 + seed % 6
        E = 8 + seed % 15
        g = aml_synth.tiny_random(n, E, 10 + seed % 7, seed, self_loops=(seed % 3 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, n, lib=lib)
        want = brute_counts(g.src, g.dst, g.ts, COLS)
        if not np.array_equal(og.count_all(COLS, threads=1), want):
            return True
        if not np.array_equal(og.count_edges(COLS, np.arange(E), threads=1), want):
            return True
    return False


@pytest.mark.parametrize("name,orig,mutated", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(orig, mutated))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-I", os.path.dirname(SRC), "-o", str(so), str(path)])
    lib = oracle.load_library(str(so))
    assert _pins_reject(lib), f"mutant {name} survived the pins"


def test_unmutated_oracle_passes(tmp_path):
    assert not _pins_reject(oracle._load())
    assert not _program_pins_reject(oracle._load())


def _program_pins_reject(lib) -> bool:
    for seed in range(6):
        n = 3 + seed % 4
        g = aml_synth.tiny_random(n, 11 + seed % 3, 8 + seed % 5, 500 + seed,
                                  self_loops=(seed % 2 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, n, lib=lib)
        for name in sorted(NOVEL):
            stages, agg = NOVEL[name]
            for delta in (0, 3, 1000):
                want = brute_program(g.src, g.dst, g.ts, stages, agg, delta)
                if not np.array_equal(og.program_count(stages, agg, delta, threads=1), want):
                    return True
    return False


@pytest.mark.parametrize("name,orig,mutated", PROGRAM_MUTANTS, ids=[m[0] for m in PROGRAM_MUTANTS])
def test_program_pins_reject_mutant(tmp_path, name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(orig, mutated))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-I", os.path.dirname(SRC), "-o", str(so), str(path)])
    lib = oracle.load_library(str(so))
    assert _program_pins_reject(lib), f"mutant {name} survived the program pins"


# mistakes in the amount constraints, caught by the amount-program pins
AMOUNT_MUTANTS = [
    ("amt-ratio-b-side-from-reach", "if (!pg_amount_ok(c, s, fb, fa)) continue;",
     "if (!pg_amount_ok(c, s, fb, ra)) continue;"),
    ("amt-range-open-below",
     "if ((s->amount_flags & OG_AMT_RANGE) && !(a >= s->amount_min && a <= s->amount_max)) return 0;",
     "if ((s->amount_flags & OG_AMT_RANGE) && !(a > s->amount_min && a <= s->amount_max)) return 0;"),
    ("amt-ratio-ignored", "  if (s->amount_flags & OG_AMT_RATIO) {\n    const double b",
     "  if (0) {\n    const double b"),
    ("amt-trigger-range-ignored",
     "        continue;  /* not a trigger */", "        ;  /* not a trigger */"),
]


def _amount_pins_reject(lib) -> bool:
    for seed in range(8):
        g = aml_synth.tiny_random(4, 12, 9, 3000 + seed)
        rng = np.random.default_rng(seed)
        src = np.concatenate([g.src, [0, 1, 2, 0, 0, 1, 2]]).astype(np.int32)
        dst = np.concatenate([g.dst, [1, 2, 0, 1, 2, 3, 3]]).astype(np.int32)
        ts = np.concatenate([g.ts, np.sort(rng.integers(0, 8, 3)),
                             np.sort(rng.integers(0, 8, 2)), np.sort(rng.integers(4, 12, 2))])
        amount = np.concatenate([rng.choice(AMOUNT_VALUES, 12), [100.0, 95.0, 90.0],
                                 [100.0, 100.0], [95.0, 95.0]]).astype(np.float32)
        og = oracle.OracleGraph(src, dst, ts, 4, lib=lib, amount=amount)
        for name in sorted(AMOUNT_PROGRAMS):
            stages, agg = AMOUNT_PROGRAMS[name]
            for delta in (3, 1000):
                want = brute_program(src, dst, ts, stages, agg, delta, amount=amount)
                if not np.array_equal(og.program_count(stages, agg, delta, threads=1), want):
                    return True
    return False


@pytest.mark.parametrize("name,orig,mutated", AMOUNT_MUTANTS, ids=[m[0] for m in AMOUNT_MUTANTS])
def test_amount_pins_reject_mutant(tmp_path, name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(orig, mutated))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-I", os.path.dirname(SRC), "-o", str(so), str(path)])
    lib = oracle.load_library(str(so))
    assert _amount_pins_reject(lib), f"mutant {name} survived the amount pins"


def test_unmutated_oracle_passes_amount_pins():
    assert not _amount_pins_reject(oracle._load())


# mistakes in the SETS aggregate (distinct edge sets of the instances),
# caught by the brute-force set pins
SETS_MUTANTS = [
    ("sets-no-dedupe", "      if (i > 0 && pg_cmp_set(r - width, r, &width) == 0) continue;\n", ""),
    ("sets-unsorted", "      for (; j > 0 && r[j - 1] > c->edges[i]; --j) r[j] = r[j - 1];\n", ""),
    ("sets-compare-short", "  for (int i = 0; i < *(const int*)width; ++i)",
     "  for (int i = 0; i + 1 < *(const int*)width; ++i)"),
    ("sets-repeat-edges", "        if (c->edges[i] == c->edges[j]) return;\n", ""),
]


def _sets_pins_reject(lib) -> bool:
    from paper_2604_12241_b300 import patterns as P
    import dataclasses
    programs = [NOVEL["fan_pairs"][0], NOVEL["common_out"][0], NOVEL["path3"][0]]
    programs += [[dataclasses.astuple(s) for s in P.scatter_gather_n(n, 0).stages] for n in (2, 3)]
    for seed in range(6):
        n = 3 + seed % 4
        g = aml_synth.tiny_random(n, 12 + seed % 3, 8 + seed % 5, 900 + seed,
                                  self_loops=(seed % 2 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, n, lib=lib)
        for stages in programs:
            for delta in (3, 1000):
                want = brute_program(g.src, g.dst, g.ts, stages, oracle.AGG_SETS, delta)
                got = og.program_count(stages, oracle.AGG_SETS, delta, threads=1)
                if not np.array_equal(got, want):
                    return True
    return False


@pytest.mark.parametrize("name,orig,mutated", SETS_MUTANTS, ids=[m[0] for m in SETS_MUTANTS])
def test_sets_pins_reject_mutant(tmp_path, name, orig, mutated):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(orig, mutated))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-I", os.path.dirname(SRC), "-o", str(so), str(path)])
    lib = oracle.load_library(str(so))
    assert _sets_pins_reject(lib), f"mutant {name} survived the set pins"


def test_unmutated_oracle_passes_sets_pins():
    assert not _sets_pins_reject(oracle._load())
