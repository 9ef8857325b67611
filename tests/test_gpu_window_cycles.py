"""Window cycles (CYCW_k: simple k-cycles within delta, edges in any time
order; Sec. 4's cycles with anticipatory edges) through the C ABI against
the CPU oracle, bit-exact: multi-tile random graphs with timestamp ties,
tiny-10k at 24 hours and 7 days beside the ordered columns, one to three
windows counted in one search, the closing-range scan and its binary-search
form, graph replay, and the refusal of incremental counting."""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import from_oracle_columns, oracle_columns

pytestmark = pytest.mark.gpu

DAY, WEEK = P.DAY, P.WEEK


def _mine(graph, pats, **kw):
    import torch
    ps = aml.PatternSet(pats)
    out = aml.mine(graph, ps, **kw)
    torch.cuda.synchronize()
    graph.sync()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed,cols", [
    (1, [("cycw", 3, 60), ("cycw", 4, 60), ("cycw", 5, 80), ("cycw", 6, 80)]),
    (2, [("cycw", 3, 30), ("cycw", 3, 90), ("cycw", 4, 200), ("cyc", 3, 200), ("cyc", 4, 90),
         ("sg", 40), ("gs", 30)]),
    (3, [("cycw", 5, 25), ("cycw", 4, 50), ("cycw", 3, 100), ("cycw", 7, 100)]),
])
def test_random_graphs_match_oracle(seed, cols):
    g = aml_synth.tiny_random(300, 20_000, 3_000, 700 + seed, self_loops=True)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(cols)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes)
    pats = from_oracle_columns(cols)
    assert (want > 0).any(axis=0).all()
    np.testing.assert_array_equal(_mine(graph, pats), want)
    before = graph.tuning()
    try:
        graph.set_tuning(close_scan_max=0)       # every closing by binary search
        np.testing.assert_array_equal(_mine(graph, pats), want)
        graph.set_tuning(own_max=0, block=64)
        np.testing.assert_array_equal(_mine(graph, pats, use_graph=True), want)
    finally:
        graph.set_tuning(**before)


def test_tiny10k_beside_ordered_columns():
    g = aml_synth.workload("tiny-10k")
    cols = ([("cycw", k, d) for d in (DAY, WEEK) for k in (3, 4, 5)]
            + oracle_columns(P.standard(DAY)))
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(cols)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    got = _mine(graph, from_oracle_columns(cols))
    np.testing.assert_array_equal(got, want)
    # planted ordered cycles on fresh accounts are window cycles too
    for m in g.motifs:
        if m.kind == "cyc" and m.fresh:
            assert (got[m.edges, cols.index(("cycw", m.k, DAY))] == 1).all()


def test_stream_refuses_window_cycles():
    ps = aml.PatternSet([P.window_cycle(3, DAY)])
    with pytest.raises(aml.AmlError) as ei:
        aml.Stream(ps, n_nodes=100, resident_window=DAY, mem_budget=1 << 26)
    assert ei.value.name == "AML_EUNSUPPORTED"
