"""Launch modes and tunables change no count: CUDA-graph replay, every
extreme of every tunable (lane vs warp work split, bucket size, closing scan
vs search, block size) and the autotuner's choice all reproduce the plain
mine bit for bit."""
import numpy as np
import pytest

import aml_synth
import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import patterns as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    g = aml_synth.workload("tiny-10k")
    graph = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True)
    ps = aml.PatternSet(P.standard(P.DAY) + P.standard(P.WEEK))
    ref = aml.mine(graph, ps).cpu().numpy()
    return graph, ps, ref


def test_graph_mode_replays_are_exact(setup):
    import torch
    graph, ps, ref = setup
    out = torch.empty(ref.shape, dtype=torch.int32, device="cuda")
    for _ in range(4):
        out.fill_(-1)
        aml.mine(graph, ps, out=out, use_graph=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    graph.sync()


@pytest.mark.parametrize("kw", [dict(own_max=0), dict(own_max=4096), dict(own_max=1),
                                dict(sg_bucket_mean=16), dict(sg_bucket_mean=512),
                                dict(close_scan_max=0), dict(close_scan_max=4096),
                                dict(block=64), dict(block=512)])
def test_tunables_do_not_change_counts(setup, kw):
    graph, ps, ref = setup
    before = graph.tuning()
    try:
        graph.set_tuning(**kw)
        np.testing.assert_array_equal(aml.mine(graph, ps).cpu().numpy(), ref)
        np.testing.assert_array_equal(aml.mine(graph, ps, use_graph=True).cpu().numpy(), ref)
    finally:
        graph.set_tuning(**before)


def test_tuning_rejects_out_of_range(setup):
    graph, _, _ = setup
    for kw in (dict(block=100), dict(sg_bucket_mean=4096), dict(own_max=-1)):
        with pytest.raises(aml.AmlError) as ei:
            graph.set_tuning(**kw)
        assert ei.value.name == "AML_EINVAL"


def test_autotune_keeps_counts(setup):
    graph, ps, ref = setup
    best, ms = aml.autotune(graph, ps, repeats=2)
    assert ms > 0 and graph.tuning() == best
    np.testing.assert_array_equal(aml.mine(graph, ps).cpu().numpy(), ref)


def test_async_host_output_and_overlapped_graphs(setup):
    """AML_MINE_HOST_ASYNC: the copy back is only enqueued; after a stream
    sync the pinned buffer holds the device result.  Two graphs on two
    streams, each destroyed while the other's work is in flight (destroy
    waits for its own streams only), give identical counts.  A pageable
    buffer is refused."""
    import torch
    graph, ps, ref = setup
    g = aml_synth.workload("tiny-10k")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.empty(ref.shape, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
            for _ in range(2)]
    live = [None, None]
    for k in range(5):
        i = k % 2
        if live[i] is not None:
            live[i].close()
            np.testing.assert_array_equal(outs[i], ref.view(np.uint32))
        outs[i][:] = 0xFFFFFFFF
        gg = aml.Graph(g.src, g.dst, g.ts, g.n_nodes, assume_sorted=True, stream=streams[i])
        aml.mine(gg, ps, out=outs[i], host_output=True, host_async=True, stream=streams[i])
        live[i] = gg
    for i in range(2):
        live[i].close()
        np.testing.assert_array_equal(outs[i], ref.view(np.uint32))
    with pytest.raises(aml.AmlError) as ei:
        aml.mine(graph, ps, out=np.empty(ref.shape, dtype=np.uint32), host_output=True,
                 host_async=True)
    assert ei.value.name == "AML_EINVAL"
