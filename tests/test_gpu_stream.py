"""Streaming recount: after every append, every resident row equals the
oracle's count over everything appended so far (bit-exact; the oracle's
canonical enumeration of the prefix, or its edge-centric query on a sample
of resident rows for the larger shapes) and the count of a full GPU mine of
the prefix, for random batch sizes, ties across batch boundaries, and
eviction; the window graph the stream updates from append to append equals
a fresh build of the same window, array by array; bad batches are refused
without changing the stream."""
import numpy as np
import pytest

import aml_synth
import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import oracle_columns

pytestmark = pytest.mark.gpu


def full_mine(g, n, pats):
    graph = aml.Graph(g.src[:n], g.dst[:n], g.ts[:n], g.n_nodes, assume_sorted=True)
    out = aml.mine(graph, aml.PatternSet(pats)).cpu().numpy().view(np.uint32)
    graph.close()
    return out


def oracle_prefix(g, n, pats):
    """The oracle's counts of every edge of the first n edges."""
    og = oracle.OracleGraph(g.src[:n], g.dst[:n], g.ts[:n], g.n_nodes)
    return og.count_all(oracle_columns(pats))


def check_resident(st, g, n, pats, want_gpu=None):
    """Resident rows equal the oracle over the prefix (and a full GPU mine,
    when given)."""
    inf = st.info()
    r0, nr = inf["resident_first_row"], inf["resident_rows"]
    assert r0 + nr == n
    got = st.read(r0, nr)
    np.testing.assert_array_equal(got, oracle_prefix(g, n, pats)[r0:r0 + nr])
    if want_gpu is not None:
        np.testing.assert_array_equal(got, want_gpu[r0:r0 + nr])
    return r0


def check_resident_sample(st, g, n, pats, rng, n_random=3000, n_hub=600):
    """Larger shapes: a sample of resident rows (random, the top hubs'
    edges, the last batch's first rows) against the oracle's edge-centric
    query over the prefix."""
    inf = st.info()
    r0, nr = inf["resident_first_row"], inf["resident_rows"]
    src, dst = g.src[:n], g.dst[:n]
    out_deg = np.bincount(src, minlength=g.n_nodes)
    in_deg = np.bincount(dst, minlength=g.n_nodes)
    hub = np.isin(src, np.argsort(out_deg)[-10:]) | np.isin(dst, np.argsort(in_deg)[-10:])
    hub_rows = np.nonzero(hub[r0:])[0] + r0
    ids = np.unique(np.concatenate([
        rng.choice(np.arange(r0, n), min(n_random, nr), replace=False),
        rng.choice(hub_rows, min(n_hub, hub_rows.size), replace=False),
        np.arange(max(r0, n - 200), n), np.arange(r0, min(n, r0 + 50))]))
    og = oracle.OracleGraph(src, dst, g.ts[:n], g.n_nodes)
    want = og.count_edges(oracle_columns(pats), ids)
    rows = st.read(r0, nr)[ids - r0]
    np.testing.assert_array_equal(rows, want)


@pytest.mark.parametrize("window_days", [8, 30])
def test_stream_equals_full_mine(window_days):
    import torch
    assert torch.cuda.is_available()
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY) + P.standard(P.WEEK)
    ps = aml.PatternSet(pats)
    st = aml.Stream(ps, g.n_nodes, resident_window=window_days * P.DAY, mem_budget=1 << 30)
    rng = np.random.default_rng(window_days)
    pos, n_checks, evicted_checks = 0, 0, 0
    E = g.n_edges
    while pos < E:
        n = int(min(E - pos, rng.integers(1, 6000)))
        info = st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n],
                         g.amount[pos:pos + n])
        assert info["first_row"] == pos and info["n_rows"] == n
        # the window graph kept between appends equals a fresh build
        assert st.check_graph() == 0
        pos += n
        if rng.random() < 0.3 or pos == E:
            r0 = check_resident(st, g, pos, pats, full_mine(g, pos, pats))
            n_checks += 1
            evicted_checks += r0 > 0
    assert n_checks >= 3
    if window_days == 8:
        assert evicted_checks >= 2   # mid-stream checks after eviction too
    inf = st.info()
    if window_days == 8:
        assert inf["resident_first_row"] > 0          # eviction happened
        with pytest.raises(aml.AmlError):
            st.read(0, 1)
    assert inf["final_end_row"] <= inf["resident_first_row"] + inf["resident_rows"]
    st.close()


def test_stream_refuses_bad_batches():
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY)
    ps = aml.PatternSet(pats)
    st = aml.Stream(ps, g.n_nodes, resident_window=2 * P.DAY, mem_budget=1 << 28)
    st.append(g.src[:1000], g.dst[:1000], g.ts[:1000])
    # late: starts before the latest appended timestamp
    with pytest.raises(aml.AmlError) as ei:
        st.append(g.src[:10], g.dst[:10], g.ts[:10])
    assert ei.value.name == "AML_ELATE"
    # decreasing inside the batch
    ts = g.ts[1000:1010].copy()
    ts[5] = ts[9] + 1
    with pytest.raises(aml.AmlError) as ei:
        st.append(g.src[1000:1010], g.dst[1000:1010], ts)
    assert ei.value.name == "AML_EUNSORTED"
    # an id outside [0, n_nodes)
    bad = g.dst[1000:1010].copy()
    bad[3] = g.n_nodes
    with pytest.raises(aml.AmlError) as ei:
        st.append(g.src[1000:1010], bad, g.ts[1000:1010])
    assert ei.value.name == "AML_EINVAL"
    # over the budget: refused, and the stream is unchanged afterwards
    cap = st.info()["capacity_rows"]
    big = 1000 + cap + 10
    if big <= g.n_edges:
        with pytest.raises(aml.AmlError) as ei:
            st.append(g.src[1000:big], g.dst[1000:big], g.ts[1000:big])
        assert ei.value.name == "AML_EADMIT"
    st.append(g.src[1000:3000], g.dst[1000:3000], g.ts[1000:3000])
    check_resident(st, g, 3000, pats, full_mine(g, 3000, pats))
    st.close()


def test_stream_hi_medium_shape_at_tenth_scale():
    """The serving configuration's shape (Zipf 1.05, hubs, 20 columns, a
    7-day resident window) at a tenth of its size: batches of log-uniform
    size in [1e3, 1e5]; the resident rows equal a full mine at the end."""
    g = aml_synth.workload("hi-medium", scale=0.1)
    pats = P.workload_patterns("hi-medium")
    ps = aml.PatternSet(pats)
    st = aml.Stream(ps, g.n_nodes, resident_window=7 * P.DAY, mem_budget=8 << 30)
    rng = np.random.default_rng(5)
    pos, E, mid = 0, g.n_edges, None
    while pos < E:
        n = int(min(E - pos, np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n],
                  g.amount[pos:pos + n])
        pos += n
        if rng.random() < 0.2:
            assert st.check_graph() == 0
        if mid is None and pos > E // 2 and st.info()["resident_first_row"] > 0:
            check_resident_sample(st, g, pos, pats, rng)   # mid-stream, after eviction
            mid = pos
    assert mid is not None
    assert st.check_graph() == 0
    inf = st.info()
    r0, nr = inf["resident_first_row"], inf["resident_rows"]
    assert r0 > 0 and r0 + nr == E
    want = full_mine(g, E, pats)
    np.testing.assert_array_equal(st.read(r0, nr), want[r0:r0 + nr])
    check_resident_sample(st, g, E, pats, rng)
    st.close()


def test_stream_graph_update_edge_cases():
    """Self-loops, repeated counterparties, equal timestamps across batch
    boundaries, single-edge batches, a batch of self-loops only, and a gap
    longer than the window (every kept row leaves): the graph updated from
    append to append equals a fresh build, and the counts a full mine."""
    from types import SimpleNamespace
    rng = np.random.default_rng(11)
    N, E = 40, 6000
    src = rng.integers(0, N, E).astype(np.int32)
    dst = rng.integers(0, N, E).astype(np.int32)
    loops = rng.random(E) < 0.05
    dst[loops] = src[loops]
    dst[2000:2010] = src[2000:2010]            # this batch holds self-loops only
    ts = (np.cumsum(rng.integers(0, 3, E)) * 60).astype(np.int32)  # many equal times
    ts[3000:] += 20 * P.DAY                    # a gap longer than every window
    assert np.all(np.diff(ts) >= 0)
    g = SimpleNamespace(src=src, dst=dst, ts=ts, n_nodes=N)
    pats = P.standard(P.DAY) + P.standard(P.WEEK)
    st = aml.Stream(aml.PatternSet(pats), N, resident_window=8 * P.DAY, mem_budget=1 << 28)
    cuts = [0, 1, 2, 3, 700, 701, 1500, 2000, 2010, 2011, 2999, 3000, 3001, 4200, 5999, E]
    for a, b in zip(cuts[:-1], cuts[1:]):
        st.append(src[a:b], dst[a:b], ts[a:b])
        assert st.check_graph() == 0, (a, b)
        if b in (1, 3, 701, 2010, 2011, 3001, 4200, E):
            check_resident(st, g, b, pats, full_mine(g, b, pats) if b in (2011, 3001, E)
                           else None)
    st.close()


def test_stream_uses_both_leg_emissions():
    """A batch with few destinations takes the delta leg emission (old legs
    only through the marked slots of batch destinations), a batch whose
    destinations take most slots the full walk; both recounts equal a full
    mine."""
    from paper_2604_12241_b300 import _lib
    g = aml_synth.workload("hi-medium", scale=0.1)
    pats = P.workload_patterns("hi-medium")
    st = aml.Stream(aml.PatternSet(pats), g.n_nodes, resident_window=7 * P.DAY,
                    mem_budget=8 << 30)
    pos = int(np.searchsorted(g.ts, 8 * P.DAY))
    st.append(g.src[:pos], g.dst[:pos], g.ts[:pos], g.amount[:pos])
    seen = set()
    for n in (50, 60000, 300, 120000, 1):
        _lib.profile_read(reset=True)
        _lib.profile_enable(True)
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n],
                  g.amount[pos:pos + n])
        _lib.profile_enable(False)
        seen |= {k for k in _lib.profile_read(reset=True) if k.startswith("k_leg_emit")}
        pos += n
    assert seen == {"k_leg_emit", "k_leg_emit_delta"}, seen
    want = full_mine(g, pos, pats)
    inf = st.info()
    r0, nr = inf["resident_first_row"], inf["resident_rows"]
    np.testing.assert_array_equal(st.read(r0, nr), want[r0:r0 + nr])
    check_resident_sample(st, g, pos, pats, np.random.default_rng(9))
    assert st.check_graph() == 0
    st.close()


@pytest.mark.parametrize("kind", ["no_sg", "trailing_only", "cycles_only"])
def test_stream_column_subsets(kind):
    """Pattern sets without scatter-gather columns (the delta leg emission
    then walks no marked slots), with trailing-window columns only (no leg
    pass at all), and with cycles only: the resident rows equal a full mine
    after appends with eviction."""
    g = aml_synth.workload("tiny-10k")
    if kind == "no_sg":
        pats = [p for p in P.standard(P.DAY) + P.standard(P.WEEK) if not p.name.startswith("SG")]
    elif kind == "trailing_only":
        pats = [P.deg_out(P.DAY), P.fan_in(P.WEEK), P.fan_out(P.DAY)]
    else:
        pats = [P.cycle(k, P.DAY) for k in (2, 3, 4)] + [P.cycle(3, P.WEEK)]
    st = aml.Stream(aml.PatternSet(pats), g.n_nodes, resident_window=8 * P.DAY,
                    mem_budget=1 << 30)
    rng = np.random.default_rng(17)
    pos, E = 0, g.n_edges
    while pos < E:
        n = int(min(E - pos, rng.integers(1, 9000)))
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n])
        pos += n
    assert check_resident(st, g, E, pats, full_mine(g, E, pats)) > 0
    assert st.check_graph() == 0
    st.close()


def test_stream_batches_at_the_one_block_sort_limit():
    """Batches of up to 16,384 edges are sorted by one block in shared
    memory, larger ones by radix passes: batches on both sides of the limit
    (and of the power of two below it) give the same window graph as a fresh
    build and the same counts as a full mine."""
    g = aml_synth.workload("tiny-10k")
    pats = P.standard(P.DAY)
    st = aml.Stream(aml.PatternSet(pats), g.n_nodes, resident_window=30 * P.DAY,
                    mem_budget=1 << 30)
    pos, E = 0, g.n_edges
    for n in (16384, 16385, 8192, 8193, 1, 2049):
        st.append(g.src[pos:pos + n], g.dst[pos:pos + n], g.ts[pos:pos + n])
        pos += n
        assert st.check_graph() == 0
    st.append(g.src[pos:], g.dst[pos:], g.ts[pos:])
    assert st.check_graph() == 0
    check_resident(st, g, E, pats, full_mine(g, E, pats))
    st.close()
