"""Scatter-gather groups too large for one hash bucket's pair loop.

A few (source, destination) account pairs joined through hundreds of
intermediaries, with parallel edges on both hops and times spread over five
days, give groups of hundreds of legs: their buckets overflow to the large
shared-memory table, where groups above 64 legs are counted by sorting
(the partner count of a leg from start and end times, minus the legs through
its own intermediary).  Background edges put small groups into the same
buckets.  Checked in full against the oracle at one, two and three SG
windows (the smaller windows counted inside the largest one's pass) and with
the other columns of the pass."""
import numpy as np
import pytest

import oracle
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P
from colmap import from_oracle_columns

pytestmark = pytest.mark.gpu

HOUR, DAY, WEEK = 3600, P.DAY, P.WEEK


def hub_graph(seed):
    rng = np.random.default_rng(seed)
    src, dst = [], []
    n_nodes = 4000
    # (s, d, intermediaries, time range of their edges)
    pairs = [(0, 1, 300, 5 * DAY), (2, 3, 200, DAY), (4, 5, 80, 3 * HOUR)]
    ts = []
    mid = 10
    for s, d, k, span in pairs:
        for _ in range(k):
            m = mid
            mid += 1
            for _ in range(int(rng.integers(1, 4))):
                src.append(s)
                dst.append(m)
                ts.append(int(rng.integers(0, span)))
            for _ in range(int(rng.integers(1, 4))):
                src.append(m)
                dst.append(d)
                ts.append(int(rng.integers(0, span)))
    n_bg = 20_000
    src += list(rng.integers(0, n_nodes, size=n_bg))
    dst += list(rng.integers(0, n_nodes, size=n_bg))
    ts += list(rng.integers(0, 5 * DAY, size=n_bg))
    return (np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32),
            np.asarray(ts, dtype=np.int32), n_nodes)


@pytest.mark.parametrize("cols", [
    [("sg", WEEK)],
    [("sg", DAY), ("sg", WEEK), ("gs", WEEK), ("cyc", 3, WEEK)],
    [("sg", HOUR), ("sg", DAY), ("sg", WEEK), ("gs", DAY)],
])
def test_large_sg_groups_match_oracle(cols):
    import torch
    src, dst, ts, n = hub_graph(11)
    want = oracle.OracleGraph(src, dst, ts, n).count_all(cols)
    g = aml.Graph(src, dst, ts, n)
    ps = aml.PatternSet(from_oracle_columns(cols))
    got = aml.mine(g, ps)
    torch.cuda.synchronize()
    g.sync()
    got = got.cpu().numpy().view(np.uint32)
    assert want[:, 0].max() > 100          # the hub groups are really there
    np.testing.assert_array_equal(got, want)
    g.close()


def huge_group_graph(seed):
    """Two (source, destination) pairs joined through 2,500 and 1,800
    intermediaries with two edges on each hop: groups of thousands of legs,
    whose buckets hold more records than the large shared-memory table
    (4,096) and are compared pair by pair, their records spread over every
    block of the launch."""
    rng = np.random.default_rng(seed)
    src, dst, ts = [], [], []
    mid = 10
    for s, d, k in ((0, 1, 2500), (2, 3, 1800)):
        for _ in range(k):
            m = mid
            mid += 1
            for _ in range(2):
                src.append(s)
                dst.append(m)
                ts.append(int(rng.integers(0, 2 * DAY)))
                src.append(m)
                dst.append(d)
                ts.append(int(rng.integers(0, 2 * DAY)))
    n_nodes = mid + 1000
    n_bg = 20_000
    src += list(rng.integers(0, n_nodes, size=n_bg))
    dst += list(rng.integers(0, n_nodes, size=n_bg))
    ts += list(rng.integers(0, 2 * DAY, size=n_bg))
    return (np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32),
            np.asarray(ts, dtype=np.int32), n_nodes)


@pytest.mark.parametrize("cols", [[("sg", WEEK)], [("sg", DAY), ("sg", WEEK)]])
def test_sg_buckets_beyond_the_large_table_match_oracle(cols):
    import torch
    src, dst, ts, n = huge_group_graph(12)
    want = oracle.OracleGraph(src, dst, ts, n).count_all(cols)
    g = aml.Graph(src, dst, ts, n)
    ps = aml.PatternSet(from_oracle_columns(cols))
    got = aml.mine(g, ps)
    torch.cuda.synchronize()
    g.sync()
    got = got.cpu().numpy().view(np.uint32)
    assert want[:, -1].max() > 4096        # a group larger than the large table
    np.testing.assert_array_equal(got, want)
    g.close()
