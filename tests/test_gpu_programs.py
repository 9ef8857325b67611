"""The generic interpretation of stage programs on the GPU against the
oracle's (og_program_count), bit-exact: programs no family matches, every
family's own program forced through the interpreter, and pattern sets that
mix interpreted and family columns; tiny random graphs with ties and
self-loops, and the tiny-10k workload.  The interpreter's refusals
(captured mines, streams, the work limit) are errors, not wrong counts."""
import dataclasses

import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from programs import AMOUNT_PROGRAMS, AMOUNT_VALUES, NOVEL, F, T, OUT, NONE, SPAN, EDGES
from colmap import oracle_columns

pytestmark = pytest.mark.gpu


def _tuples(pattern):
    return [dataclasses.astuple(s) for s in pattern.stages]


def _mine(g, pats):
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=getattr(g, "amount", None))
    out = aml.mine(graph, aml.PatternSet(pats)).cpu().numpy().view(np.uint32)
    graph.close()
    return out


def _family_programs(delta):
    out = [P.deg_out(delta), P.fan_in(delta), P.gather_scatter(delta, mirrored=True),
           P.scatter_gather(delta), P.scatter_gather(delta, trigger="gather")]
    for k in (2, 3, 4):
        out.append(P.cycle(k, delta))
    out += [P.cycle(4, delta, closing="intersect"), P.window_cycle(3, delta)]
    return [P.interpreted(p) for p in out]


def test_novel_programs_are_interpreted():
    ps = aml.PatternSet([P.program(st, agg, 5) for st, agg in NOVEL.values()])
    assert all(c["family"] == 8 and c["name"].startswith("PROGRAM") for c in ps.columns)


@pytest.mark.parametrize("seed", range(6))
def test_programs_match_oracle_on_tiny_graphs(seed):
    g = aml_synth.tiny_random(4 + seed % 5, 60 + 20 * seed, 30, 300 + seed,
                              self_loops=(seed % 2 == 0))
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    for delta in (0, 7, 1000):
        pats = [P.program(st, agg, delta) for st, agg in NOVEL.values()]
        pats += _family_programs(delta)
        got = _mine(g, pats)
        for j, p in enumerate(pats):
            want = og.program_count(_tuples(p), p.aggregate, p.delta, threads=4)
            np.testing.assert_array_equal(got[:, j], want,
                                          err_msg=f"column {j} ({p.name}), delta {delta}")


def test_programs_match_oracle_with_a_hub():
    """A hub holding a third of the edges: its triggers have hundreds of
    first-stage candidates and go to the warp-per-trigger walk."""
    from types import SimpleNamespace
    rng = np.random.default_rng(42)
    E, N = 800, 30
    src = rng.integers(0, N, E).astype(np.int32)
    dst = rng.integers(0, N, E).astype(np.int32)
    hub = rng.random(E) < 0.3
    src[hub & (rng.random(E) < 0.5)] = 0
    dst[hub & (src != 0)] = 0
    ts = np.sort(rng.integers(0, 200, E)).astype(np.int32)
    g = SimpleNamespace(src=src, dst=dst, ts=ts, n_nodes=N)
    og = oracle.OracleGraph(src, dst, ts, N)
    assert max(np.bincount(src, minlength=N)[0], np.bincount(dst, minlength=N)[0]) > 100
    for delta in (50, 1000):
        pats = [P.program(st, agg, delta) for st, agg in NOVEL.values()]
        pats += _family_programs(delta) + [P.scatter_gather_n(3, delta),
                                           P.scatter_gather_nodes(delta)]
        got = _mine(g, pats)
        for j, p in enumerate(pats):
            want = og.program_count(_tuples(p), p.aggregate, p.delta, threads=8)
            np.testing.assert_array_equal(got[:, j], want,
                                          err_msg=f"column {j} ({p.name}), delta {delta}")


def test_programs_match_oracle_on_tiny10k():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    pats = [P.program(st, agg, P.DAY) for st, agg in NOVEL.values()]
    pats += _family_programs(P.DAY)
    pats += [P.scatter_gather_n(n, P.DAY) for n in (3, 4)]  # "at least N" intermediaries
    pats += [P.scatter_gather_nodes(P.DAY)]                      # node-level SG
    pats += [P.gather_scatter_n(2, 2, P.DAY), P.gather_scatter_n(3, 1, P.DAY)]
    # family columns beside the interpreted ones in the same mine
    fam = P.standard(P.DAY)
    got = _mine(g, pats + fam)
    for j, p in enumerate(pats):
        want = og.program_count(_tuples(p), p.aggregate, p.delta)
        np.testing.assert_array_equal(got[:, j], want, err_msg=p.name or f"program {j}")
    want_fam = og.count_all(oracle_columns(fam))
    np.testing.assert_array_equal(got[:, len(pats):], want_fam)
    # interpreted family programs reproduce their families (SG twice over)
    names = [p.name for p in pats]
    sg = got[:, names.index(f"SG@{P.DAY}")]
    np.testing.assert_array_equal(sg.astype(np.uint64),
                                  want_fam[:, 5].astype(np.uint64) * 2)


def test_interpreted_columns_are_refused_where_unsupported():
    import torch
    g = aml_synth.tiny_random(10, 200, 50, 3)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes)
    st, agg = NOVEL["path3"]
    ps = aml.PatternSet([P.program(st, agg, 20)])
    out = torch.zeros((g.n_edges, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(aml.AmlError) as ei:
        aml.mine(graph, ps, out=out, use_graph=True)
    assert ei.value.name == "AML_EUNSUPPORTED"
    with pytest.raises(aml.AmlError) as ei:
        aml.Stream(ps, g.n_nodes, resident_window=100)
    assert ei.value.name == "AML_EUNSUPPORTED"
    graph.close()


def test_work_limit_ends_the_launch_with_an_error():
    """Seven nested loops over ~5,000 parallel edges per node: far more than
    2^34 candidate visits.  The launch stops at the limit and the call
    reports it; the graph stays usable."""
    rng = np.random.default_rng(1)
    E, N = 20000, 4
    src = rng.integers(0, N, E).astype(np.int32)
    dst = ((src + 1 + rng.integers(0, N - 1, E)) % N).astype(np.int32)
    ts = np.sort(rng.integers(0, 1000, E)).astype(np.int32)
    graph = aml.Graph(src, dst, ts, N)
    chain = [T] + [F(v, OUT, v + 1, NONE, SPAN) for v in range(1, 8)]
    with pytest.raises(aml.AmlError) as ei:
        aml.mine(graph, aml.PatternSet([P.program(chain, EDGES, 10**6)]))
    assert ei.value.name == "AML_EUNSUPPORTED" and "limit" in str(ei.value)
    # the graph still mines normally afterwards
    out = aml.mine(graph, aml.PatternSet([P.deg_out(100)])).cpu().numpy().view(np.uint32)
    og = oracle.OracleGraph(src, dst, ts, N)
    np.testing.assert_array_equal(out[:, 0], og.count_all([("deg_out", 100)])[:, 0])
    graph.close()


def test_amount_programs_match_oracle():
    """Amount ranges and ratios: tiny graphs with planted motifs whose
    amounts meet the ratio bounds exactly, and tiny-10k with its lognormal
    amounts."""
    from types import SimpleNamespace
    cases = []
    for seed in range(4):
        base = aml_synth.tiny_random(6, 120, 40, 4000 + seed, self_loops=(seed == 1))
        rng = np.random.default_rng(seed)
        src = np.concatenate([base.src, [0, 1, 2, 0, 0, 1, 2]]).astype(np.int32)
        dst = np.concatenate([base.dst, [1, 2, 0, 1, 2, 3, 3]]).astype(np.int32)
        ts = np.concatenate([base.ts, np.sort(rng.integers(0, 20, 3)),
                             np.sort(rng.integers(0, 20, 2)),
                             np.sort(rng.integers(10, 30, 2))]).astype(np.int32)
        amount = np.concatenate([rng.choice(AMOUNT_VALUES, 120), [100.0, 95.0, 90.0],
                                 [100.0, 100.0], [95.0, 95.0]]).astype(np.float32)
        cases.append((SimpleNamespace(src=src, dst=dst, ts=ts, n_nodes=6, amount=amount),
                      (5, 1000)))
    cases.append((aml_synth.workload("tiny-10k"), (P.DAY,)))
    for g, deltas in cases:
        og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount)
        for delta in deltas:
            pats = [P.program(st, agg, delta, name=n) for n, (st, agg) in AMOUNT_PROGRAMS.items()]
            got = _mine(g, pats)
            for j, p in enumerate(pats):
                want = og.program_count(_tuples(p), p.aggregate, p.delta)
                np.testing.assert_array_equal(got[:, j], want, err_msg=f"{p.name}, delta {delta}")


def test_amount_constraints_are_validated():
    bad = [P.program([T, F(1, OUT, 2, NONE, SPAN) + (1, 5.0, 1.0, 0.0, 0.0)], EDGES, 10),
           P.program([T + (2, 0.0, 0.0, 0.5, 1.0), F(1, OUT, 2, NONE, SPAN)], EDGES, 10),
           P.program([T, F(1, OUT, 2, NONE, SPAN) + (4, 0.0, 0.0, 0.0, 0.0)], EDGES, 10)]
    for p in bad:
        with pytest.raises(aml.AmlError) as ei:
            aml.PatternSet([p])
        assert ei.value.name == "AML_EINVAL"
    # any amount constraint sends a family program to the interpreter
    st = [dataclasses.astuple(s) for s in P.gather_scatter(10).stages]
    st[1] = st[1][:9] + (1, 0.0, 1e9, 0.0, 0.0)
    assert aml.PatternSet([P.program(st, P.AGG_INSTANCES, 10)]).columns[0]["family"] == 8


def test_programs_match_oracle_on_hi_small():
    """Full size, every row: hi-small (5,078,345 edges) with its amounts, a
    3-hop path, an intersection program, interpreted GS and an amount
    program, in one mine as the bench runs them."""
    g = aml_synth.workload("hi-small")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount)
    pats = [P.program(*NOVEL["path3"], P.DAY), P.program(*NOVEL["common_out"], P.DAY),
            P.interpreted(P.gather_scatter(P.DAY)),
            P.program(*AMOUNT_PROGRAMS["fee_forward"], P.DAY)]
    got = _mine(g, pats)
    for j, p in enumerate(pats):
        want = og.program_count(_tuples(p), p.aggregate, p.delta)
        np.testing.assert_array_equal(got[:, j], want, err_msg=f"column {j}")


def test_programs_in_every_cycle_mode():
    """Interpreted columns beside family columns give the same counts in the
    plain, persistent and learned cycle modes (the interpreter runs after
    the cycle search, whichever form it takes)."""
    g = aml_synth.workload("tiny-10k")
    pats = (P.standard(P.DAY) + [P.program(*NOVEL["path3"], P.DAY),
                                 P.program(*NOVEL["distinct_2hop"], P.DAY)])
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes)
    ps = aml.PatternSet(pats)
    outs = [aml.mine(graph, ps, mode=m).cpu().numpy() for m in ("plain", "persistent", "learned")]
    graph.close()
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])


def _exact_sg(delta):
    """Exact-size scatter-gather bins: n = 2 by the SG family and through the
    interpreter, n = 3 and 4 through the interpreter (ordered count / n!)."""
    return [P.scatter_gather_exact(2, delta), P.scatter_gather_exact(2, delta, interpret=True),
            P.scatter_gather_exact(3, delta), P.scatter_gather_exact(4, delta)]


@pytest.mark.parametrize("seed", range(4))
def test_exact_size_scatter_gathers_match_oracle_on_tiny_graphs(seed):
    """The SETS columns against the oracle's distinct edge sets, on dense
    small graphs with ties, parallel edges and self-loops."""
    rng = np.random.default_rng(600 + seed)
    n, E = 7 + seed, 90 + 20 * seed
    src = rng.integers(0, n, E).astype(np.int32)
    dst = rng.integers(0, n, E).astype(np.int32)
    ts = rng.integers(0, 40, E).astype(np.int32)
    from types import SimpleNamespace
    g = SimpleNamespace(src=src, dst=dst, ts=ts, n_nodes=n)
    og = oracle.OracleGraph(src, dst, ts, n)
    reached = 0
    for delta in (3, 8, 40):
        pats = _exact_sg(delta)
        got = _mine(g, pats)
        for j, p in enumerate(pats):
            want = og.program_count(_tuples(p), oracle.AGG_SETS, delta, threads=4)
            np.testing.assert_array_equal(got[:, j], want, err_msg=f"{p.name}, delta {delta}")
        reached += int((got[:, 3] > 0).sum())
    assert reached > 0  # 4-intermediary motifs occur


def test_exact_size_scatter_gathers_match_oracle_on_tiny10k():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    pats = _exact_sg(P.DAY) + P.standard(P.DAY)
    got = _mine(g, pats)
    for j, p in enumerate(pats[:4]):
        want = og.program_count(_tuples(p), oracle.AGG_SETS, p.delta)
        np.testing.assert_array_equal(got[:, j], want, err_msg=p.name)
        assert want.any(), p.name
    np.testing.assert_array_equal(got[:, 4:], og.count_all(oracle_columns(P.standard(P.DAY))))


# ---- the stacked bipartite ("Stack", Sec. 8): SETS = bindings / 8 ----

@pytest.mark.parametrize("seed", range(3))
def test_stack_matches_oracle_on_dense_graphs(seed):
    """The interpreter's per-binding count divided by the 8 bindings of every
    instance, against the oracle's distinct edge sets, on dense small graphs
    (parallel edges, ties, self-loops)."""
    rng = np.random.default_rng(9300 + seed)
    n, E = 7 + seed, 60 + 20 * seed
    src = rng.integers(0, n, E).astype(np.int32)
    dst = rng.integers(0, n, E).astype(np.int32)
    ts = rng.integers(0, 20, E).astype(np.int32)
    from types import SimpleNamespace
    g = SimpleNamespace(src=src, dst=dst, ts=ts, n_nodes=n)
    og = oracle.OracleGraph(src, dst, ts, n)
    reached = 0
    for delta in (3, 8, 40):
        p = P.stack(delta)
        got = _mine(g, [p])[:, 0]
        want = og.program_count(_tuples(p), oracle.AGG_SETS, delta, threads=4)
        np.testing.assert_array_equal(got, want, err_msg=f"delta {delta}")
        reached += int((want > 0).sum())
    assert reached > 0


def test_stack_matches_oracle_on_tiny10k():
    g = aml_synth.workload("tiny-10k")
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    pats = [P.stack(P.DAY), P.stack(3 * 3600)] + P.standard(P.DAY, 3)
    got = _mine(g, pats)
    for j, p in enumerate(pats[:2]):
        want = og.program_count(_tuples(p), oracle.AGG_SETS, p.delta)
        np.testing.assert_array_equal(got[:, j], want, err_msg=p.name)
    assert got[:, 0].any()
    np.testing.assert_array_equal(got[:, 2:], og.count_all(oracle_columns(P.standard(P.DAY, 3))))
