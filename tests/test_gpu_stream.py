"""Walks streamed to host memory chunk by chunk (the output side of FN-Multi,
Section 3.4) give the rows of one n2v_walk call over the whole id range.

The chunks do not divide the range (a ragged last chunk), the ring has one to
three slots (one slot: no overlap; more: a chunk computes while the previous
one is copied), and the copies run on their own stream or on the compute
stream.  Needs a GB300.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.mark.parametrize("variant", ["persistent", "plain"])
@pytest.mark.parametrize("slots", [1, 2, 3])
def test_streamed_rows_equal_one_call(variant, slots):
    wl = G.WORKLOADS["er"]
    g = G.workload_graph("er")
    graph = n2v.Graph.from_csr(g)
    starts = np.arange(g.n, dtype=np.int32)
    p, q = wl.pq[0]
    want = n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, variant).cpu()
    got = n2v.walk_to_host(graph, starts, wl.r, wl.l, p, q, wl.seed, ring_walks=7777, ring_slots=slots,
                           variant=variant)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    assert got.is_pinned() and torch.equal(got, want)
    ids = np.arange(0, g.n * wl.r, 97)
    rows = oracle.walk(g.row_ptr, g.col, None, starts, wl.l, p, q, wl.seed, ids, threads=8)
    np.testing.assert_array_equal(got.numpy()[ids], rows)
    graph.close()


def test_streamed_sub_range_weighted_on_one_stream():
    g = G.with_weights(G.rmat(14, 16, 0.57, 0.19, 0.19, 4), 6, 1, 100)
    graph = n2v.Graph.from_csr(g)
    starts = np.arange(g.n, dtype=np.int32)
    want = n2v.walk(graph, starts, 3, 30, 1.0, 0.5, 9, "persistent", walk_begin=1000, walk_count=40_000).cpu()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        got = n2v.walk_to_host(graph, starts, 3, 30, 1.0, 0.5, 9, ring_walks=4096, ring_slots=2, walk_begin=1000,
                               walk_count=40_000, stream=side, copy_stream=None)
    assert torch.equal(got, want)
    graph.close()


def test_streaming_argument_checks():
    g = G.er(1000, 4000, 2)
    graph = n2v.Graph.from_csr(g)
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    host = torch.empty((g.n, 10), dtype=torch.int32).pin_memory()
    ring = torch.empty((2, 256, 10), dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
    for slots, variant in [(0, n2v.N2V_PERSISTENT), (9, n2v.N2V_PERSISTENT),
                           (2, n2v.N2V_PERSISTENT | n2v.N2V_FLAG_CUDA_GRAPH)]:
        with pytest.raises(n2v.N2VError) as e:
            n2v.n2v_walk_stream(graph.handle, starts, g.n, 1, 10, 1.0, 1.0, 1, 0, g.n, host, ring, 256, slots, ws,
                                variant)
        assert e.value.code == n2v.N2V_ERR_INVALID_ARG
    graph.close()
