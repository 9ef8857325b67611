"""The fused persistent mine (AML_MINE_FUSED): a window's leg pass (leg
count, leg offsets, leg emission) and every level of its cycle search in one
cooperative launch whose warps take tiles of work from queues and whose
blocks meet at grid-wide barriers.  Its counts equal
the oracle's and the plain mine's, replayed from a captured CUDA graph too,
on tiny-10k, on a hub graph, on graphs with fewer edges than the launch has
blocks, on pattern sets without cycles, and at hi-small's full size (sampled
oracle rows, every row against the plain mine); the fused launch replaces the
separate leg and cycle kernels; a barrier wait that runs out (wait limit 0)
ends the launch with AML_ETIMEOUT at aml_sync and leaves the context usable."""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import oracle_columns

pytestmark = pytest.mark.gpu


def _mine(graph, ps, **kw):
    return aml.mine(graph, ps, **kw).cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("kmax", [3, 5, 7])
def test_fused_equals_oracle_tiny_10k(kmax):
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY, kmax) + P.standard(P.WEEK, kmax)
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(oracle_columns(pats))
    for _ in range(3):   # the first learns the level sizes with the plain search
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
    for _ in range(3):
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused", use_graph=True), want)
    graph.sync()
    graph.close()


def test_fused_launch_replaces_leg_and_cycle_kernels():
    from paper_2604_12241_b300 import _lib
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY, 5)
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(oracle_columns(pats))
    np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)  # learns the sizes
    graph.sync()
    _lib.profile_enable(True)
    try:
        _lib.profile_read(reset=True)
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
        graph.sync()
        ran = _lib.profile_read(reset=True)
    finally:
        _lib.profile_enable(False)
    assert ran.get("k_mine_fused", (0, 0.0))[0] == 1, ran
    for k in ("k_leg_count", "k_leg_emit", "k_cyc_level", "k_cyc_emit", "k_cyc_fused"):
        assert k not in ran, ran
    assert "k_sg_bucket" in ran and "k_assemble" in ran
    graph.close()


@pytest.mark.parametrize("n_edges", [1, 37, 700, 5000])
def test_fused_with_fewer_edges_than_blocks(n_edges):
    """Fewer edge tiles than the launch has warps, and chunks of zero or one
    edge for the offsets: most blocks of the launch count and emit nothing
    but still meet every barrier."""
    rng = np.random.default_rng(n_edges)
    N = max(4, n_edges // 6)
    src = rng.integers(0, N, n_edges).astype(np.int32)
    dst = rng.integers(0, N, n_edges).astype(np.int32)
    ts = np.sort(rng.integers(0, 3 * 3600, n_edges)).astype(np.int32)
    pats = P.standard(3600, 5)
    ps = aml.PatternSet(pats)
    graph = aml.Graph(src, dst, ts, N, assume_sorted=True)
    want = oracle.OracleGraph(src, dst, ts, N).count_all(oracle_columns(pats))
    for _ in range(3):
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
    np.testing.assert_array_equal(_mine(graph, ps, mode="fused", use_graph=True), want)
    graph.sync()
    graph.close()


def test_fused_without_cycles():
    """GS, SG and 2-cycles only: the launch ends after the leg emission."""
    g = aml_synth.workload("tiny-10k")
    pats = [p for p in P.standard(P.DAY, 2) + P.standard(P.WEEK, 2)]
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(oracle_columns(pats))
    assert want[:, [p.name.startswith("SG") for p in pats]].sum() > 0
    for _ in range(3):
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
    np.testing.assert_array_equal(_mine(graph, ps, mode="fused", use_graph=True), want)
    graph.sync()
    graph.close()


def test_fused_with_two_leg_passes():
    """A 24-hour window with longer cycles than the 7-day one gets a leg
    pass (and a fused launch) of its own; the second launch finds the
    accumulators already zeroed by the first and runs beside the first
    window's SG grouping."""
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY, 5) + P.standard(P.WEEK, 3)
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(oracle_columns(pats))
    for _ in range(3):
        np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
    np.testing.assert_array_equal(_mine(graph, ps, mode="fused", use_graph=True), want)
    graph.sync()
    graph.close()


def test_fused_on_hub_graph():
    """A few accounts with most of the edges: long child lists written by
    whole warps, and chunks of the frontier that start inside one path's
    children."""
    rng = np.random.default_rng(3)
    N, E = 60, 20_000
    w = 1.0 / np.arange(1, N + 1) ** 0.8      # the top account holds ~15% of the edges
    w /= w.sum()
    src = rng.choice(N, E, p=w).astype(np.int32)
    dst = rng.choice(N, E, p=rng.permutation(w)).astype(np.int32)
    ts = np.sort(rng.integers(0, 2 * P.DAY, E)).astype(np.int32)
    pats = [P.cycle(k, 900) for k in (3, 4, 5, 6)]
    ps = aml.PatternSet(pats)
    graph = aml.Graph(src, dst, ts, N, assume_sorted=True)
    want = oracle.OracleGraph(src, dst, ts, N).count_all(oracle_columns(pats))
    assert (want.sum(axis=0) > 100).all()
    for kw in (dict(own_max=0), dict(own_max=4096), dict(own_max=16)):
        graph.set_tuning(**kw)
        for _ in range(2):
            np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), want)
    graph.sync()
    graph.close()


def test_fused_hi_small_full_size():
    import torch
    g = aml_synth.workload("hi-small")
    pats = P.workload_patterns("hi-small")
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, amount=g.amount, assume_sorted=True)
    plain = aml.mine(graph, ps)
    aml.mine(graph, ps, mode="fused")
    fused = aml.mine(graph, ps, mode="fused", use_graph=True)
    assert torch.equal(fused, plain)
    rng = np.random.default_rng(8)
    motif = np.concatenate([m.edges for m in g.motifs])
    ids = np.unique(np.concatenate([rng.choice(g.n_edges, 3000, replace=False), motif]))
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_edges(oracle_columns(pats),
                                                                         ids)
    rows = fused[torch.from_numpy(ids).cuda()].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(rows, want)
    graph.sync()
    graph.close()


def test_barrier_wait_that_runs_out_reports_etimeout():
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.WEEK, 6)
    ps = aml.PatternSet(pats)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    ref = _mine(graph, ps)
    _mine(graph, ps, mode="fused")          # learns the level sizes
    graph.sync()
    graph.set_wait_limit(0)                 # every barrier gives up unless already complete
    seen = False
    for _ in range(3):
        aml.mine(graph, ps, mode="fused")
        try:
            graph.sync()
        except aml.AmlError as err:
            assert err.name == "AML_ETIMEOUT"
            seen = True
            break
    assert seen
    graph.set_wait_limit(1 << 32)
    np.testing.assert_array_equal(_mine(graph, ps, mode="fused"), ref)
    np.testing.assert_array_equal(_mine(graph, ps), ref)
    graph.sync()
    with pytest.raises(aml.AmlError) as ei:
        graph.set_wait_limit(-1)
    assert ei.value.name == "AML_EINVAL"
    graph.close()
