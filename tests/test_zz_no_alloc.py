"""The allocation-free entry point (n2v_walk_noalloc) gives n2v_walk's rows.

n2v_walk_noalloc serves callers that cannot allocate device memory (code
inside a memory pool or arena owned by another runtime, plugins given only a
stream and their buffers): it runs the persistent sampler on a scratch array
inside the library instead of a caller workspace.  Its rows must equal those
of n2v_walk on the same inputs, call after call, because the scratch keeps
the previous call's contents.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.  It also passes alone in a
fresh process: the first call on the device sets up the scratch address.
"""
import numpy as np
import pytest
import torch

from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_matches_n2v_walk_on_two_calls(weighted):
    g = G.rmat(14, 16, 0.57, 0.19, 0.19, 11)
    if weighted:
        g = G.with_weights(g, 5, 1, 100)
    graph = n2v.Graph.from_csr(g)
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    r, l, p, q, seed = 3, 40, 0.5, 2.0, 21
    W = g.n * r
    want = n2v.walk(graph, starts, r, l, p, q, seed, "persistent")  # caller workspace path
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    for call in range(2):  # the second call runs on the scratch the first one left behind
        out = torch.full((W, l), -7, dtype=torch.int32, device="cuda")
        n2v.n2v_walk_noalloc(graph.handle, starts, g.n, r, l, p, q, seed, 0, W, out)
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
        assert torch.equal(out, want), f"call {call}: rows differ from n2v_walk"
    graph.close()


def test_noalloc_sub_range_and_rejected_size():
    g = G.rmat(12, 16, 0.57, 0.19, 0.19, 3)
    graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(chunk_walkers=64))
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    # r = 10 walks from each of the 4096 vertices: ids [100, 20100) of 40960
    want = n2v.walk(graph, starts, 10, 10, 2.0, 0.5, 9, "persistent", walk_begin=100, walk_count=20_000)
    out = torch.empty_like(want)
    n2v.n2v_walk_noalloc(graph.handle, starts, g.n, 10, 10, 2.0, 0.5, 9, 100, 20_000, out)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    assert torch.equal(out, want)
    # 64 walks per launch: 40,000 walks would need more launch counters than the scratch holds
    big = torch.empty((40_000, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(n2v.N2VError) as e:
        n2v.n2v_walk_noalloc(graph.handle, starts, g.n, 10, 10, 2.0, 0.5, 9, 0, 40_000, big)
    assert e.value.code == n2v.N2V_ERR_NO_MEM
    graph.close()


def test_noalloc_specials_beyond_the_scratch_spill():
    """On K_800 every step at v from t has 799 special neighbours (t and every other vertex
    but v).  With 32 shared-memory slots per warp and the spill area the 4 MiB scratch leaves
    each warp (a few hundred slots at the default grid), the specials of every step overflow
    both and are enumerated again segment by segment; the rows must still equal n2v_walk's
    (which keeps them all in its 4096-slot workspace spill) and the oracle's."""
    import oracle

    k = 800
    edges = [(i, j) for i in range(k) for j in range(i + 1, k)]
    g = G.from_edges(k, edges)
    tune = n2v.default_tune(smem_specials=32, thread_max_deg=0)
    graph = n2v.Graph.from_csr(g, tune=tune)
    _, blocks, threads = n2v.n2v_launch_shape(graph.handle)
    per_warp = ((4 << 20) - 4096) // 4 // (blocks * threads // 32)
    assert k - 1 > 32 + per_warp, "the clique no longer overflows the scratch spill"
    starts = torch.arange(k, dtype=torch.int32, device="cuda")
    r, l, p, q, seed = 8, 12, 0.5, 2.0, 31
    W = k * r
    want = n2v.walk(graph, starts, r, l, p, q, seed, "persistent")
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    for call in range(2):
        out = torch.full((W, l), -7, dtype=torch.int32, device="cuda")
        n2v.n2v_walk_noalloc(graph.handle, starts, k, r, l, p, q, seed, 0, W, out)
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
        assert torch.equal(out, want), f"call {call}: rows differ from n2v_walk"
    ids = np.arange(0, W, 7)
    rows = oracle.walk(g.row_ptr, g.col, None, np.arange(k, dtype=np.int32), l, p, q, seed, ids, threads=8)
    np.testing.assert_array_equal(want[torch.from_numpy(ids).cuda()].cpu().numpy(), rows)
    graph.close()
