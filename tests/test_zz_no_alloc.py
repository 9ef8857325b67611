"""aml_fan_noalloc: the FAN column computed with no device allocation.

Some callers cannot call cudaMalloc where they need the feature (inside a
CUDA stream capture, under a fixed pre-reserved memory budget, or in a loop
that cannot take an allocator's synchronization).  This checks, through the
C ABI, that the allocation-free entry point gives exactly aml_mine's FAN
columns, on two calls in a row (the fixed scratch array keeps the previous
call's contents), and that graphs above its scratch limit are refused.
This file is collected last so a failure here leaves every other result in.
"""
import ctypes

import numpy as np
import pytest

import aml_synth
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import _lib, patterns as P

pytestmark = pytest.mark.gpu


def _call(graph, delta, direction, out, stream):
    return _lib.lib().aml_fan_noalloc(graph.handle, delta, direction,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))


def test_fan_noalloc_matches_mine_twice():
    import torch
    assert torch.cuda.is_available()
    g = aml_synth.workload("tiny-10k")
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    stream = torch.cuda.current_stream()
    out = torch.full((g.n_edges,), -1, dtype=torch.int32, device="cuda")
    cases = [(P.DIR_OUT, P.fan_out), (P.DIR_IN, P.fan_in)]
    for delta in (P.DAY, P.WEEK, 0):
        for direction, fam in cases:
            ref = aml.mine(graph, aml.PatternSet([fam(delta)]))[:, 0].clone()
            for _ in range(2):
                out.fill_(-1)
                assert _call(graph, delta, direction, out, stream) == 0, \
                    _lib.lib().aml_last_error()
                torch.cuda.synchronize()
                np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    graph.sync()


def test_fan_noalloc_refuses_graphs_above_its_limit():
    import torch
    g = aml_synth.tiny_random(50_000, 4_300_000, 86400 * 5, seed=77)
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes)
    assert graph.info()["n_list_edges"] > 4_194_304
    out = torch.empty((g.n_edges,), dtype=torch.int32, device="cuda")
    rc = _call(graph, 86400, P.DIR_OUT, out, torch.cuda.current_stream())
    assert _lib.STATUS[rc] == "AML_EINVAL"
    assert b"4,194,304" in _lib.lib().aml_last_error()


def test_fan_noalloc_at_its_limit():
    """A graph with exactly 4,194,304 non-loop edges: 2,048 tiles, so the
    single-block scan of the tile totals is full, and the last tile is a
    whole one; and one edge fewer, so the last tile is partial."""
    import torch
    stream = torch.cuda.current_stream()
    for n_edges, direction, fam in ((4_194_304, P.DIR_OUT, P.fan_out),
                                    (4_194_303, P.DIR_IN, P.fan_in)):
        g = aml_synth.tiny_random(50_000, n_edges, 86400 * 5, seed=78)
        graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes)
        assert graph.info()["n_list_edges"] == n_edges
        ref = aml.mine(graph, aml.PatternSet([fam(P.DAY)]))[:, 0].clone()
        out = torch.full((g.n_edges,), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            out.fill_(-1)
            assert _call(graph, P.DAY, direction, out, stream) == 0, \
                _lib.lib().aml_last_error()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        graph.sync()
        graph.close()
