"""GPU sampler vs CPU oracle: bit-exact walks through the C ABI (needs a GB300).

Walks are integer results (vertex ids chosen by integer prefix sums under a
fixed Philox stream), so the bar is bit-exact equality of every compared row.
Every variant (plain, binned, persistent, persistent recorded as a CUDA graph)
and every tuning that changes which code path runs (thread vs warp bins, the
shared-memory spill path, the hub hash sets, chunked launches) must give the
oracle's rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v
from small_graphs import big_star, small_graphs, two_hubs

pytestmark = pytest.mark.gpu

VARIANTS = ["plain", "binned", "persistent"]

TUNES = {
    "default": {},
    "all_warp": dict(thread_max_deg=0),
    "all_thread": dict(thread_max_deg=1 << 30),
    "spill": dict(thread_max_deg=0, smem_specials=32, spill_specials=64),
    "hubs": dict(thread_max_deg=0, hub_count=4096, hub_min_degree=2, stream_ratio=0),
    "chunks": dict(chunk_walkers=1000, block_threads=128),
    "probe": dict(thread_max_deg=0, stream_ratio=0),
    # every list longer than 64 staged through many 64-element TMA windows
    "stage": dict(thread_max_deg=0, stream_ratio=100_000, stage_window=64),
    "stage4": dict(thread_max_deg=0, stream_ratio=100_000, stage_window=64, stage_buffers=4),
    # specials kept 32 at a time: the enumeration restarts segment by segment
    "segments": dict(thread_max_deg=0, smem_specials=32, spill_specials=0, stage_window=64, stream_ratio=100_000),
    # the persistent kernel's other register budgets: 16, 24 and 32 resident warps per SM
    "warps16": dict(blocks_per_sm=4),
    "warps24": dict(block_threads=256, blocks_per_sm=3),
    "warps32": dict(blocks_per_sm=8, stage_window=512),
    # rank bitmaps on every vertex of degree >= 2 (up to 64): the probe modes through one-load lookups
    "bitmaps": dict(thread_max_deg=0, bitmap_hubs=64, hub_min_degree=2),
    "bitmaps_segments": dict(thread_max_deg=0, bitmap_hubs=64, hub_min_degree=2, smem_specials=32, spill_specials=0),
    # the persistent sampler's block batches: every step on the whole block (threshold 1), none (2^30),
    # and the block tier through each generator and the segment path
    "block_all": dict(thread_max_deg=0, block_min_deg=1),
    "block_none": dict(block_min_deg=1 << 30),
    "block_stage": dict(thread_max_deg=0, block_min_deg=1, stream_ratio=100_000, stage_window=64),
    "block_probe": dict(thread_max_deg=0, block_min_deg=1, stream_ratio=0),
    "block_segments": dict(thread_max_deg=0, block_min_deg=1, smem_specials=32, spill_specials=0, stage_window=64,
                           stream_ratio=100_000),
    "block_bitmaps": dict(thread_max_deg=0, block_min_deg=1, bitmap_hubs=64, hub_min_degree=2),
    # the merge form for every step whose lists fit a window (1024, and 64 for ragged windows), and never
    "merge_all": dict(thread_max_deg=0, merge_ratio=1_000_000),
    "merge_w64": dict(thread_max_deg=0, merge_ratio=1_000_000, stage_window=64),
    "merge_off": dict(thread_max_deg=0, merge_ratio=0),
    "block_merge": dict(thread_max_deg=0, merge_ratio=1_000_000, block_min_deg=1, stage_window=64),
    # the persistent sampler's launches with a persisting L2 window over the start of col
    "l2persist": dict(l2_persist_mb=8),
}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()
    yield
    torch.cuda.synchronize()


def gpu_rows(g, starts, r, l, p, q, seed, variant, tune=None, walk_begin=0, walk_count=None, cuda_graph=False,
             graph=None):
    G_ = graph if graph is not None else n2v.Graph.from_csr(g, tune=n2v.default_tune(**(tune or {})))
    out = n2v.walk(G_, starts, r, l, p, q, seed, variant, walk_begin=walk_begin, walk_count=walk_count,
                   cuda_graph=cuda_graph)
    assert n2v.n2v_stream_status(G_.handle) == n2v.N2V_OK
    return out.cpu().numpy()


def oracle_rows(g, starts, l, p, q, seed, ids, threads=8):
    return oracle.walk(g.row_ptr, g.col, g.w, np.asarray(starts, np.int32), l, p, q, seed,
                       np.asarray(ids, np.int64), threads=threads)


# --------------------------------------------------------------------------
# small graphs: every variant x every tuning, full rows

SMALL = small_graphs()
SMALL_CASES = [(nm, pq) for nm in SMALL for pq in [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25), (3.0, 0.7)]]


@pytest.mark.parametrize("name,pq", SMALL_CASES, ids=[f"{a}-{b[0]}-{b[1]}" for a, b in SMALL_CASES])
def test_small_graphs_every_variant_and_tuning(name, pq):
    g = SMALL[name]
    p, q = pq
    starts = np.arange(g.n, dtype=np.int32)
    r, l = 37, 9  # walk count not a multiple of 32
    want = oracle_rows(g, starts, l, p, q, 5, np.arange(g.n * r))
    for tname, tune in TUNES.items():
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**tune))
        for v in VARIANTS:
            got = gpu_rows(g, starts, r, l, p, q, 5, v, graph=graph)
            np.testing.assert_array_equal(got, want, err_msg=f"{name} {tname} {v}")


# --------------------------------------------------------------------------
# the Erdos-Renyi workload: G(n=1e4, m=1e5), r=10, l=80, p=0.5, q=2, full output

@pytest.fixture(scope="module")
def er():
    wl = G.WORKLOADS["er"]
    g = G.workload_graph("er")
    starts = np.arange(g.n, dtype=np.int32)
    p, q = wl.pq[0]
    want = oracle_rows(g, starts, wl.l, p, q, wl.seed, np.arange(g.n * wl.r))
    return g, starts, wl, want


@pytest.mark.parametrize("variant", VARIANTS)
def test_er_full_output(er, variant):
    g, starts, wl, want = er
    p, q = wl.pq[0]
    got = gpu_rows(g, starts, wl.r, wl.l, p, q, wl.seed, variant)
    np.testing.assert_array_equal(got, want)


def test_er_cuda_graph_replay(er):
    g, starts, wl, want = er
    p, q = wl.pq[0]
    graph = n2v.Graph.from_csr(g)
    # the legacy default stream cannot be recorded
    with pytest.raises(n2v.N2VError):
        n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, "persistent", cuda_graph=True, stream=0)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(2):  # record, then replay
            got = gpu_rows(g, starts, wl.r, wl.l, p, q, wl.seed, "persistent", cuda_graph=True, graph=graph)
            np.testing.assert_array_equal(got, want)
        got = gpu_rows(g, starts, wl.r, wl.l, p, q, wl.seed, "plain", cuda_graph=True, graph=graph)
        np.testing.assert_array_equal(got, want)


def test_er_traffic_matches_oracle(er):
    g, starts, wl, want = er
    graph = n2v.Graph.from_csr(g)
    walks = torch.from_numpy(want).cuda()
    assert n2v.traffic(graph, starts, 0, walks) == oracle.traffic(g.row_ptr, False, starts,
                                                                  np.arange(want.shape[0]), want)


def test_weighted_traffic_matches_oracle():
    g = G.with_weights(G.rmat(12, 16, 0.57, 0.19, 0.19, 8), 3, 1, 100)
    graph = n2v.Graph.from_csr(g)
    starts = np.arange(g.n, dtype=np.int32)
    walks = n2v.walk(graph, starts, 3, 30, 0.5, 2.0, 5, "persistent")
    got = n2v.traffic(graph, starts, 0, walks)
    want = oracle.traffic(g.row_ptr, True, starts, np.arange(walks.shape[0]), walks.cpu().numpy())
    assert got == want and got[2] < got[1]


def test_split_ranges_equal_whole(er):
    """Any split of the walk-id range (chunking, sharding) gives the same rows."""
    g, starts, wl, want = er
    p, q = wl.pq[0]
    graph = n2v.Graph.from_csr(g)
    total = g.n * wl.r
    cuts = [0, 1, 33, 40_000, 77_777, total]
    for v in VARIANTS:
        parts = [gpu_rows(g, starts, wl.r, wl.l, p, q, wl.seed, v, walk_begin=a, walk_count=b - a, graph=graph)
                 for a, b in zip(cuts[:-1], cuts[1:])]
        np.testing.assert_array_equal(np.concatenate(parts), want)


# --------------------------------------------------------------------------
# R-MAT graphs

@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("pq", [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25)])
def test_rmat14_full_output(weighted, pq):
    g = G.rmat(14, 16, 0.57, 0.19, 0.19, 3)
    if weighted:
        g = G.with_weights(g, 9, 1, 100)
    p, q = pq
    starts = np.arange(g.n, dtype=np.int32)
    want = oracle_rows(g, starts, 20, p, q, 77, np.arange(g.n * 2))
    for tname in ["default", "hubs", "spill", "probe", "stage", "stage4", "segments", "warps16", "warps24", "warps32",
                  "bitmaps", "bitmaps_segments", "block_all", "block_none", "block_stage", "block_probe",
                  "block_segments", "block_bitmaps", "merge_all", "merge_w64", "merge_off", "block_merge",
                  "l2persist"]:
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**TUNES[tname]))
        for v in VARIANTS:
            got = gpu_rows(g, starts, 2, 20, p, q, 77, v, graph=graph)
            np.testing.assert_array_equal(got, want, err_msg=f"{tname} {v}")


def sample_ids(g, n_starts, r, k, seed):
    """k random walk ids plus every walk that starts at one of the 64 largest hubs."""
    rng = np.random.default_rng(seed)
    ids = rng.choice(n_starts * r, size=min(k, n_starts * r), replace=False)
    hubs = np.argsort(-g.degrees())[:64]
    hub_ids = (np.arange(r)[:, None] * n_starts + hubs[None, :]).ravel()
    return np.unique(np.concatenate([ids, hub_ids]))


@pytest.fixture(scope="module")
def rmat20():
    g = G.workload_graph("rmat20")
    return g, n2v.Graph.from_csr(g, tune=n2v.default_tune(hub_count=1024, bitmap_hubs=32))


@pytest.mark.parametrize("pq", [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25)])
def test_rmat20_workload(rmat20, pq):
    """R-MAT scale 20 at full size: every variant agrees on the whole output, and
    sampled rows (random ids + walks from the largest hubs) match the oracle."""
    g, graph = rmat20
    wl = G.WORKLOADS["rmat20"]
    p, q = pq
    starts = np.arange(g.n, dtype=np.int32)
    outs = {v: n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, v) for v in ["binned", "persistent"]}
    # the plain sampler on the first round (every start vertex once)
    outs["plain"] = n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, "plain", walk_count=g.n)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    assert torch.equal(outs["binned"], outs["persistent"])
    assert torch.equal(outs["plain"], outs["persistent"][: g.n])
    ids = sample_ids(g, g.n, wl.r, 3000, 1)
    want = oracle_rows(g, starts, wl.l, p, q, wl.seed, ids)
    got = outs["persistent"][torch.from_numpy(ids).cuda()].cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_rmat23_weighted_workload():
    """Weighted R-MAT scale 23 (w in [1,100]), p=1, q=0.5, persistent sampler with
    the hub cache on the top 0.1% of vertices: sampled rows match the oracle."""
    wl = G.WORKLOADS["rmat23w"]
    g = G.workload_graph("rmat23w")
    graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(hub_count=g.n // 1000, bitmap_hubs=32))
    assert graph.info().hub_count > 0 and graph.info().bitmap_hubs > 0
    p, q = wl.pq[0]
    starts = np.arange(g.n, dtype=np.int32)
    out = n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, "persistent")
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    ids = sample_ids(g, g.n, wl.r, 1500, 2)
    want = oracle_rows(g, starts, wl.l, p, q, wl.seed, ids)
    got = out[torch.from_numpy(ids).cuda()].cpu().numpy()
    np.testing.assert_array_equal(got, want)


# --------------------------------------------------------------------------
# degenerate and extreme shapes

def test_long_lists_star_and_twin_hubs():
    for g in [big_star(1 << 18), two_hubs(3000, extra=50)]:
        starts = np.arange(min(g.n, 4000), dtype=np.int32)
        want = oracle_rows(g, starts, 5, 0.5, 2.0, 3, np.arange(starts.size))
        for tname in ["default", "hubs", "spill", "probe", "stage", "stage4", "segments", "bitmaps",
                      "bitmaps_segments", "block_all", "block_stage", "block_segments", "block_bitmaps", "merge_all",
                      "merge_w64", "block_merge"]:
            graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**TUNES[tname]))
            for v in VARIANTS:
                got = gpu_rows(g, starts, 1, 5, 0.5, 2.0, 3, v, graph=graph)
                np.testing.assert_array_equal(got, want, err_msg=f"{g.name} {tname} {v}")


def test_isolated_starts_and_l1():
    g = G.from_edges(6, [(0, 1), (1, 2)])  # 3, 4, 5 isolated
    starts = np.arange(6, dtype=np.int32)
    for l in (1, 3):
        want = oracle_rows(g, starts, l, 2.0, 0.5, 1, np.arange(12))
        for v in VARIANTS:
            np.testing.assert_array_equal(gpu_rows(g, starts, 2, l, 2.0, 0.5, 1, v), want)
    assert (want[3:6] == -1).all()


def test_empty_call_is_a_no_op():
    g = SMALL["und7"]
    graph = n2v.Graph.from_csr(g)
    out = torch.full((0, 4), 7, dtype=torch.int32, device="cuda")
    for v in VARIANTS:
        n2v.walk(graph, [0], 1, 4, 1.0, 1.0, 1, v, walk_begin=0, walk_count=0, out=out)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK


def test_start_out_of_range_sets_status():
    g = SMALL["und7"]
    graph = n2v.Graph.from_csr(g)
    for v in VARIANTS:
        out = n2v.walk(graph, [0, 99], 1, 4, 1.0, 1.0, 1, v)
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_ERR_INVALID_ARG
        assert (out[1] == -1).all().item()
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK  # cleared


def test_overflow_is_rejected():
    g = G.from_edges(301, [(0, i) for i in range(1, 301)], weights=[2**32 - 1] * 300)
    graph = n2v.Graph.from_csr(g)
    n2v.walk(graph, [1], 1, 3, 1.0, 1.0, 1, "persistent")  # max_wsum * 2^16 < 2^64
    with pytest.raises(n2v.N2VError) as e:
        n2v.walk(graph, [1], 1, 3, 2.0**-8, 1.0, 1, "persistent")
    assert e.value.code == n2v.N2V_ERR_OVERFLOW


@pytest.mark.parametrize("bad", ["unsorted", "duplicate", "out_of_range", "row_ptr"])
def test_invalid_graph_is_rejected(bad):
    g = SMALL["und7"]
    rp, col = g.row_ptr.copy(), g.col.copy()
    if bad == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif bad == "duplicate":
        col[1] = col[0]
    elif bad == "out_of_range":
        col[3] = 7
    else:
        rp[2], rp[3] = rp[3], rp[2]
    with pytest.raises(n2v.N2VError) as e:
        n2v.Graph(rp, col)
    assert e.value.code == n2v.N2V_ERR_INVALID_GRAPH


def test_bounded_wait_times_out_cleanly():
    """A wait that can never complete gives up after its limit, reports
    N2V_ERR_TIMEOUT through the status word, and leaves the context usable."""
    g = SMALL["und7"]
    graph = n2v.Graph.from_csr(g)
    n2v.n2v_selftest_timeout(graph.handle, 2_000_000)  # about 1 ms of SM clock
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_ERR_TIMEOUT
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK  # cleared
    starts = np.arange(g.n, dtype=np.int32)
    want = oracle_rows(g, starts, 5, 1.0, 1.0, 2, np.arange(g.n))
    np.testing.assert_array_equal(gpu_rows(g, starts, 1, 5, 1.0, 1.0, 2, "persistent", graph=graph), want)


def test_persistent_launch_shape():
    """128-thread blocks; 20 resident warps per SM by default, the tuning's count otherwise, capped by shared memory."""
    g = G.er(1000, 5000, 1)
    shapes = {}
    for name, tune in [("default", {}), ("w16", dict(blocks_per_sm=4)), ("w24", dict(block_threads=256, blocks_per_sm=3)),
                       ("w32", dict(blocks_per_sm=8, stage_window=512)), ("w32big", dict(blocks_per_sm=8))]:
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**tune))
        sms, blocks, threads = n2v.n2v_launch_shape(graph.handle)
        assert threads == 128 and blocks % sms == 0
        shapes[name] = blocks // sms
    assert shapes["default"] == 5 and shapes["w16"] == 4 and shapes["w24"] == 6 and shapes["w32"] == 8
    # 32 warps of two 1024-element windows each (9312 bytes a warp) do not fit in one SM's shared memory
    assert shapes["w32big"] < 8

