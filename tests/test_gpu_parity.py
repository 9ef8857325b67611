"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every count is an integer, so the bar is bit-exact equality.  Sizes span
several thread blocks and ragged tails; hi-small is checked at full size (the
benchmark's configuration) on an oracle-computed edge sample plus invariants
that hold at any size.
"""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import from_oracle_columns, oracle_columns

pytestmark = pytest.mark.gpu

DAY, WEEK = P.DAY, P.WEEK

SMALL_COLS = [("deg_out", 5), ("deg_in", 5), ("fan_out", 5), ("fan_in", 5), ("deg_out", 0),
              ("fan_in", 2), ("gs", 5), ("gs", 0), ("sg", 6), ("sg", 100), ("cyc", 2, 6),
              ("cyc", 3, 6), ("cyc", 4, 8), ("cyc", 5, 9), ("cyc", 3, 1000), ("cyc", 6, 1000),
              ("cyc", 7, 1000)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    aml._lib.lib()


def gpu_counts(src, dst, ts, n_nodes, pats, assume_sorted=False, amount=None):
    import torch
    g = aml.Graph(src, dst, ts, n_nodes, amount=amount, assume_sorted=assume_sorted)
    ps = aml.PatternSet(pats)
    out = aml.mine(g, ps)
    torch.cuda.synchronize()
    g.sync()
    res = out.cpu().numpy().view(np.uint32)
    g.close()
    return res


def test_random_tiny_graphs():
    pats = from_oracle_columns(SMALL_COLS)
    for seed in range(150):
        n = 3 + seed % 7
        E = 6 + seed % 30
        g = aml_synth.tiny_random(n, E, 10 + seed % 9, seed, self_loops=(seed % 3 == 0))
        want = oracle.OracleGraph(g.src, g.dst, g.ts, n).count_all(SMALL_COLS)
        got = gpu_counts(g.src, g.dst, g.ts, n, pats)
        np.testing.assert_array_equal(got, want, err_msg=f"seed {seed}")


@pytest.mark.parametrize("seed", range(4))
def test_multi_tile_random_graphs(seed):
    """~20K edges, dense ties, unsorted input, self-loops: many blocks and
    radix-sort tiles, ragged tails everywhere."""
    rng = np.random.default_rng(seed)
    n, E = 200 + 100 * seed, 15_000 + 3_001 * seed
    g = aml_synth.tiny_random(n, E, 2_000, 500 + seed, self_loops=True)
    cols = [("deg_out", 50), ("deg_in", 50), ("fan_out", 50), ("fan_in", 50), ("gs", 30),
            ("sg", 20), ("cyc", 2, 40), ("cyc", 3, 40), ("cyc", 4, 40), ("cyc", 5, 40)]
    want = oracle.OracleGraph(g.src, g.dst, g.ts, n).count_all(cols)
    got = gpu_counts(g.src, g.dst, g.ts, n, from_oracle_columns(cols))
    np.testing.assert_array_equal(got, want)
    assert rng is not None


@pytest.fixture(scope="module")
def tiny10k():
    return aml_synth.workload("tiny-10k")


def test_tiny10k_full_parity(tiny10k):
    g = tiny10k
    pats = P.standard(DAY) + P.standard(WEEK)
    want = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes).count_all(oracle_columns(pats))
    got = gpu_counts(g.src, g.dst, g.ts, g.n_nodes, pats, assume_sorted=True, amount=g.amount)
    np.testing.assert_array_equal(got, want)
    assert got[:, 5].sum() > 0 and got[:, 8].sum() > 0


def test_alternative_programs_agree(tiny10k):
    g = tiny10k
    a = [P.gather_scatter(WEEK), P.scatter_gather(WEEK)] + [P.cycle(k, WEEK) for k in (3, 4, 5)]
    b = ([P.gather_scatter(WEEK, mirrored=True), P.scatter_gather(WEEK, trigger="gather")]
         + [P.cycle(k, WEEK, closing="intersect") for k in (3, 4, 5)])
    np.testing.assert_array_equal(gpu_counts(g.src, g.dst, g.ts, g.n_nodes, a),
                                  gpu_counts(g.src, g.dst, g.ts, g.n_nodes, b))


def test_host_output_and_ld_padding(tiny10k):
    import torch
    g = tiny10k
    pats = P.standard(DAY)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    ps = aml.PatternSet(pats)
    dev = aml.mine(graph, ps).cpu().numpy().view(np.uint32)
    host = aml.mine(graph, ps, host_output=True)
    np.testing.assert_array_equal(dev, host)
    wide = torch.full((g.n_edges, 13), -7, dtype=torch.int32, device="cuda")
    aml.mine(graph, ps, out=wide)
    torch.cuda.synchronize()
    w = wide.cpu().numpy()
    np.testing.assert_array_equal(w[:, :10].view(np.uint32), dev)
    assert (w[:, 10:] == -7).all()
    again = aml.mine(graph, ps).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(again, dev)   # repeated mines are identical
    graph.sync()


def test_edge_cases():
    pats = P.standard(10)
    # no edges
    out = gpu_counts(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), 5, pats)
    assert out.shape == (0, 10)
    # only self-loops
    src = np.array([1, 1, 2], np.int32)
    out = gpu_counts(src, src, np.array([0, 1, 2], np.int32), 3, pats)
    assert not out.any()
    # one edge
    out = gpu_counts(np.array([0], np.int32), np.array([1], np.int32), np.array([5], np.int32), 2,
                     pats)
    assert out.tolist() == [[1, 1, 1, 1, 0, 0, 0, 0, 0, 0]]
    # timestamps at the int32 limits with the widest window
    big = P.standard(2**31 - 1)
    src = np.array([0, 1, 2, 0, 1], np.int32)
    dst = np.array([1, 2, 0, 2, 0], np.int32)
    ts = np.array([-2**31, 0, 2**31 - 1, -2**31 + 5, 2**31 - 2], np.int32)
    want = oracle.OracleGraph(src, dst, ts, 3).count_all(oracle_columns(big))
    np.testing.assert_array_equal(gpu_counts(src, dst, ts, 3, big), want)
    # large node ids (rows are allocated for every account)
    N = 30_000_000
    src = np.array([N - 1, 5, N - 2, N - 1], np.int32)
    dst = np.array([5, N - 2, N - 1, 5], np.int32)
    ts = np.array([1, 2, 3, 4], np.int32)
    want = oracle.OracleGraph(src, dst, ts, N).count_all(oracle_columns(pats))
    np.testing.assert_array_equal(gpu_counts(src, dst, ts, N, pats), want)


def test_input_errors():
    pats = P.standard(10)
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    with pytest.raises(aml.AmlError) as ei:
        aml.Graph(src, dst, np.array([3, 2, 1], np.int32), 3, assume_sorted=True)
    assert ei.value.name == "AML_EUNSORTED"
    with pytest.raises(aml.AmlError) as ei:
        aml.Graph(src, np.array([1, 3, 0], np.int32), np.array([1, 2, 3], np.int32), 3)
    assert ei.value.name == "AML_EINVAL"
    # the same unsorted input without the promise is accepted and sorted
    out = gpu_counts(src, dst, np.array([3, 2, 1], np.int32), 3, pats)
    want = oracle.OracleGraph(src, dst, np.array([3, 2, 1], np.int32), 3).count_all(
        oracle_columns(pats))
    np.testing.assert_array_equal(out, want)


@pytest.fixture(scope="module")
def hi_small():
    g = aml_synth.workload("hi-small")
    pats = P.workload_patterns("hi-small")
    got = gpu_counts(g.src, g.dst, g.ts, g.n_nodes, pats, assume_sorted=True, amount=g.amount)
    return g, pats, got


def _sample(g, rng, n_random=15_000):
    E = g.n_edges
    out_deg = np.bincount(g.src, minlength=g.n_nodes)
    in_deg = np.bincount(g.dst, minlength=g.n_nodes)
    hub_out = np.argsort(out_deg)[-20:]
    hub_in = np.argsort(in_deg)[-20:]
    hub_edges = np.nonzero(np.isin(g.src, hub_out) | np.isin(g.dst, hub_in))[0]
    motif = np.concatenate([m.edges for m in g.motifs])
    ids = np.concatenate([rng.choice(E, n_random, replace=False),
                          rng.choice(hub_edges, 2_000, replace=False), motif,
                          np.arange(50), np.arange(E - 50, E)])
    return np.unique(ids)


def test_hi_small_sampled_parity(hi_small):
    g, pats, got = hi_small
    ids = _sample(g, np.random.default_rng(11))
    og = oracle.OracleGraph(g.src, g.dst, g.ts, g.n_nodes)
    want = og.count_edges(oracle_columns(pats), ids)
    np.testing.assert_array_equal(got[ids], want)


def test_hi_small_invariants_and_planted(hi_small):
    g, pats, got = hi_small
    names = [p.name for p in pats]
    c = {n: i for i, n in enumerate(names)}
    x = got.astype(np.int64)
    for d in (DAY, WEEK):
        for k in range(2, 6):
            assert x[:, c[f"CYC{k}@{d}"]].sum() % k == 0
        assert x[:, c[f"SG@{d}"]].sum() % 4 == 0
        assert x[:, c[f"GS@{d}"]].sum() % 2 == 0
        assert (x[:, c[f"FAN_OUT@{d}"]] <= x[:, c[f"DEG_OUT@{d}"]]).all()
        assert (x[:, c[f"FAN_IN@{d}"]] <= x[:, c[f"DEG_IN@{d}"]]).all()
    assert (x[:, 10:] >= x[:, :10]).all()
    for m in g.motifs:
        if not m.fresh:
            continue
        rows = got[m.edges]
        if m.kind == "sg":
            assert (rows[:, c[f"SG@{DAY}"]] == m.k - 1).all()
        else:
            assert (rows[:, c[f"CYC{m.k}@{DAY}"]] == 1).all()


def test_sg_pair_larger_than_a_bucket():
    """One (s, d) pair with 1,440 legs (more than a shared-memory bucket
    holds) plus background noise: exercises the oversized-bucket path."""
    rng = np.random.default_rng(5)
    s, d, n_mid, par = 0, 1, 40, 6
    src, dst, ts = [], [], []
    for m in range(2, 2 + n_mid):
        for _ in range(par):
            src.append(s); dst.append(m); ts.append(int(rng.integers(0, 500)))
            src.append(m); dst.append(d); ts.append(int(rng.integers(500, 1000)))
    n = 2 + n_mid + 30
    for _ in range(3000):
        a, b = rng.integers(0, n, 2)
        if a != b:
            src.append(int(a)); dst.append(int(b)); ts.append(int(rng.integers(0, 3000)))
    src, dst, ts = (np.asarray(x, np.int32) for x in (src, dst, ts))
    cols = [("sg", 1000), ("sg", 200), ("gs", 1000), ("cyc", 3, 600), ("cyc", 4, 600)]
    want = oracle.OracleGraph(src, dst, ts, n).count_all(cols)
    got = gpu_counts(src, dst, ts, n, from_oracle_columns(cols))
    np.testing.assert_array_equal(got, want)
    assert got[:, 0].max() > 1000


def test_hub_rows_span_many_chunks():
    """Two hubs with ~6,000 out- and ~6,000 in-slots each (repeated
    counterparties, tied timestamps) plus background: their rows cross several
    chunks of the DEG/FAN scan, including chunks in which no row starts."""
    rng = np.random.default_rng(11)
    n = 400
    src, dst, ts = [], [], []
    for hub in (0, 1):
        for _ in range(12_000):
            c = int(rng.integers(2, 2 + 150 + 100 * hub))
            t = int(rng.integers(0, 4_000))
            if rng.random() < 0.5:
                src.append(hub); dst.append(c)
            else:
                src.append(c); dst.append(hub)
            ts.append(t)
    for _ in range(4_000):
        a, b = rng.integers(0, n, 2)
        src.append(int(a)); dst.append(int(b)); ts.append(int(rng.integers(0, 4_000)))
    src, dst, ts = (np.asarray(x, np.int32) for x in (src, dst, ts))
    cols = [(f, w) for w in (0, 7, 60, 900, 10_000)
            for f in ("deg_out", "deg_in", "fan_out", "fan_in")]
    want = oracle.OracleGraph(src, dst, ts, n).count_all(cols)
    got = gpu_counts(src, dst, ts, n, from_oracle_columns(cols))
    np.testing.assert_array_equal(got, want)
