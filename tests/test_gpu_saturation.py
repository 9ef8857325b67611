"""Saturation of the counts on the GPU, against the oracle.

Every column is an exact count saturated at the graph's count limit
(2^32-1).  No graph that fits a test reaches 2^32 instances on one edge, so
the limit is lowered through the ABI (aml_graph_set_count_limit,
aml_stream_set_count_limit) and the GPU's rows are compared with the
oracle's enumeration run under the same limit (itself pinned against
min(brute force, limit)): plain and captured mines of tiny random graphs and
of tiny-10k, and a stream whose stored rows gain instances append after
append, so that an old row's stored value plus its new instances must be
saturated, not wrapped.
"""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import from_oracle_columns, oracle_columns

pytestmark = pytest.mark.gpu

COLS = [("deg_out", 5), ("deg_in", 5), ("fan_out", 5), ("fan_in", 5), ("gs", 5), ("sg", 6),
        ("sg", 100), ("cyc", 2, 6), ("cyc", 3, 6), ("cyc", 4, 8), ("cyc", 5, 9)]


def _mine(graph, pats, use_graph=False, mode=None):
    kw = {} if mode is None else {"mode": mode}
    out = aml.mine(graph, aml.PatternSet(pats), use_graph=use_graph, **kw)
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("limit", [1, 2, 3, 7])
def test_tiny_graphs_saturate_like_the_oracle(limit):
    reached = 0
    for seed in range(16):
        n = 3 + seed % 5
        g = aml_synth.tiny_random(n, 14 + seed % 11, 6 + seed % 5, 7100 + seed,
                                  self_loops=(seed % 3 == 0))
        og = oracle.OracleGraph(g.src, g.dst, g.ts, n)
        full = og.count_all(COLS)
        want = og.count_all(COLS, limit=limit)
        np.testing.assert_array_equal(want, np.minimum(full, limit))
        graph = aml.Graph(g.src, g.dst, g.ts, n)
        graph.set_count_limit(limit)
        np.testing.assert_array_equal(_mine(graph, from_oracle_columns(COLS)), want)
        reached += int((full > limit).sum())
        graph.close()
    assert reached > 20   # the limit is really reached, on many edges


def test_tiny_10k_saturates_plain_captured_and_fused():
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY)
    cols = oracle_columns(pats)
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    full = _mine(graph, pats, use_graph=True)
    np.testing.assert_array_equal(full, og.count_all(cols))
    for limit in (3, 40):
        graph.set_count_limit(limit)   # drops the captured mine of the old bound
        want = og.count_all(cols, limit=limit)
        assert (want != og.count_all(cols)).any()
        np.testing.assert_array_equal(_mine(graph, pats), want)
        np.testing.assert_array_equal(_mine(graph, pats, use_graph=True), want)
        for _ in range(2):  # the fused mine (the first learns its sizes)
            np.testing.assert_array_equal(_mine(graph, pats, mode="fused"), want)
    graph.set_count_limit(0xFFFFFFFF)
    np.testing.assert_array_equal(_mine(graph, pats, use_graph=True), full)
    with pytest.raises(aml.AmlError):
        graph.set_count_limit(0)
    graph.close()


@pytest.mark.parametrize("limit", [2, 5])
def test_stream_old_row_add_saturates(limit):
    """Rows gain instances from later batches: each stored row is
    min(full-history count, limit) after every append."""
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY)
    cols = oracle_columns(pats)
    st = aml.Stream(aml.PatternSet(pats), g.n_nodes, resident_window=3 * P.DAY,
                    mem_budget=1 << 30)
    st.set_count_limit(limit)
    rng = np.random.default_rng(limit)
    pos, E, checks = 0, 40_000, 0
    while pos < E:
        n = int(min(E - pos, rng.integers(200, 5000)))
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n])
        pos += n
        if rng.random() < 0.35 or pos == E:
            og = oracle.OracleGraph(g.src[:pos], g.dst[:pos], g.ts[:pos], g.n_nodes)
            want = og.count_all(cols, limit=limit)
            inf = st.info()
            r0, nr = inf["resident_first_row"], inf["resident_rows"]
            np.testing.assert_array_equal(st.read(r0, nr), want[r0:r0 + nr])
            checks += 1
    assert checks >= 3
    assert st.info()["resident_first_row"] > 0   # rows were evicted on the way
    st.close()
