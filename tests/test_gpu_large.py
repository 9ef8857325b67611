"""Full-size parity on the larger workloads.

* hi-medium (2,032,095 accounts, 31,898,238 transactions, Zipf 1.05, hubs up
  to 1e5): the learned-binning configuration.  The cost model is trained on
  up to 1M anchors; the learned-binned mine equals the level-synchronous mine
  on every row, and both equal the oracle on a sample of edges.
* hi-large (2,070,980 accounts, 179,702,229 transactions over 90 days,
  cycles up to 6): the resident-graph configuration, mined with graph replay
  as the benchmark does, checked against the oracle on a sample of edges and
  against the learned-binned persistent search on every row.

Samples: random edges, edges of the top hubs, every planted motif edge, and
the first and last ids.
"""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import oracle_columns

pytestmark = pytest.mark.gpu


def _sample(g, rng, n_random, n_hub):
    E = g.n_edges
    out_deg = np.bincount(g.src, minlength=g.n_nodes)
    in_deg = np.bincount(g.dst, minlength=g.n_nodes)
    hubs = np.isin(g.src, np.argsort(out_deg)[-20:]) | np.isin(g.dst, np.argsort(in_deg)[-20:])
    hub_edges = np.nonzero(hubs)[0]
    motif = np.concatenate([m.edges for m in g.motifs])
    ids = np.concatenate([rng.choice(E, n_random, replace=False),
                          rng.choice(hub_edges, min(n_hub, hub_edges.size), replace=False),
                          motif, np.arange(50), np.arange(E - 50, E)])
    return np.unique(ids)


def _check_sample(g, pats, got_rows, ids):
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    want = og.count_edges(oracle_columns(pats), ids)
    np.testing.assert_array_equal(got_rows, want)


def test_hi_medium_learned_binning_full_size():
    import torch
    g = aml_synth.workload("hi-medium")
    pats = P.workload_patterns("hi-medium")
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount, assume_sorted=True)
    ps = aml.PatternSet(pats)
    plain = aml.mine(graph, ps, use_graph=True)
    rep = aml.cost_train(graph, ps, max_samples=1_000_000, epochs=10, seed=5)
    assert rep["n_train"] + rep["n_test"] == min(rep["n_items"], 1_000_000)
    assert np.isfinite(rep["final_train_mse"]) and rep["test_spearman"] > 0.3
    learned = aml.mine(graph, ps, mode="learned")
    assert torch.equal(learned, plain)
    del learned
    ids = _sample(g, np.random.default_rng(21), 4_000, 1_000)
    rows = plain[torch.from_numpy(ids).cuda()].cpu().numpy().view(np.uint32)
    _check_sample(g, pats, rows, ids)
    graph.close()


def test_hi_large_full_size():
    import torch
    g = aml_synth.workload("hi-large")
    pats = P.workload_patterns("hi-large")
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount, assume_sorted=True)
    ps = aml.PatternSet(pats)
    out = aml.mine(graph, ps, use_graph=True)
    assert out.shape == (g.n_edges, len(pats))
    ids = _sample(g, np.random.default_rng(22), 4_000, 1_000)
    rows = out[torch.from_numpy(ids).cuda()].cpu().numpy().view(np.uint32)
    _check_sample(g, pats, rows, ids)
    # invariants over every row
    x = out.to(torch.int64)
    names = [p.name for p in pats]
    for k in range(3, 7):
        assert int(x[:, names.index(f"CYC{k}@{P.DAY}")].sum()) % k == 0
    assert int(x[:, names.index(f"SG@{P.DAY}")].sum()) % 4 == 0
    assert bool((x[:, names.index(f"FAN_OUT@{P.WEEK}")] >=
                 x[:, names.index(f"FAN_OUT@{P.DAY}")]).all())
    del x
    aml.cost_train(graph, ps, max_samples=200_000, epochs=5, seed=6)
    learned = aml.mine(graph, ps, mode="learned")
    assert torch.equal(learned, out)
    graph.close()
