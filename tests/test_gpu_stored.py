"""Stored transition tables (the per-edge precomputation of Section 3.2, Eq. 1) on the GPU.

* The table has one entry per (edge t->v, neighbour of v): sum_e deg(col[e])
  entries, which is sum_i d_i^2 on an undirected graph (Eq. 1).
* Each edge's stored total equals the oracle's on-the-fly total T for that
  (t, v) step, and its cumulative weights are non-decreasing.
* Walks sampled from the table equal the oracle's rows (and n2v_walk's) bit
  for bit, on the small graphs, R-MAT with weights, and the ER workload.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v
from small_graphs import small_graphs

pytestmark = pytest.mark.gpu

TILE = 512 * 8  # elements per tile of the build's scan (the layout's scratch)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()
    yield
    torch.cuda.synchronize()


def up256(x):
    return (x + 255) & ~255


def table_arrays(table: n2v.StoredTable, nnz: int):
    """(off [nnz+1], cdf [entries]) read back from the documented buffer layout."""
    raw = table.buf.view(torch.uint8)
    off_at = 256
    tiles = (nnz + 1 + TILE - 1) // TILE
    sums_at = up256(off_at + 8 * (nnz + 1))
    cdf_at = up256(sums_at + 8 * tiles)
    off = raw[off_at:off_at + 8 * (nnz + 1)].view(torch.int64).cpu().numpy()
    cdf = raw[cdf_at:cdf_at + 8 * table.entries].view(torch.int64).cpu().numpy().view(np.uint64)
    return off, cdf


def entries_host(g):
    d = g.degrees()
    return int(d[g.col].astype(np.int64).sum())


def oracle_rows(g, starts, l, p, q, seed, ids):
    return oracle.walk(g.row_ptr, g.col, g.w, np.asarray(starts, np.int32), l, p, q, seed,
                       np.asarray(ids, np.int64), threads=8)


SMALL = small_graphs()


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("pq", [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25), (3.0, 0.7)])
def test_small_graphs_rows_equal_oracle(name, pq):
    g = SMALL[name]
    graph = n2v.Graph.from_csr(g)
    table = n2v.StoredTable(graph, *pq)
    assert table.entries == entries_host(g)
    starts = np.arange(g.n, dtype=np.int32)
    got = n2v.stored_walk(graph, table, starts, 50, 12, 9).cpu().numpy()
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    want = oracle_rows(g, starts, 12, pq[0], pq[1], 9, np.arange(g.n * 50))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("weighted", [False, True])
def test_table_matches_eq1_and_oracle_totals(weighted):
    g = G.rmat(12, 16, 0.57, 0.19, 0.19, 4)
    if weighted:
        g = G.with_weights(g, 5, 1, 100)
    p, q = 0.5, 2.0
    graph = n2v.Graph.from_csr(g)
    table = n2v.StoredTable(graph, p, q)
    d = g.degrees().astype(np.int64)
    # undirected: one entry per ordered pair of neighbours of each vertex, sum d_i^2 (Eq. 1)
    assert table.entries == int((d * d).sum())
    assert table.nbytes >= 8 * table.entries
    off, cdf = table_arrays(table, g.nnz)
    np.testing.assert_array_equal(off[1:] - off[:-1], d[g.col])
    a_p, a_q = oracle.alpha_q16(p, q)
    src = np.repeat(np.arange(g.n), d)
    rng = np.random.default_rng(3)
    for e in rng.choice(g.nnz, 300, replace=False):
        t, v = int(src[e]), int(g.col[e])
        C = cdf[off[e]:off[e + 1]]
        assert np.all(C[1:] >= C[:-1])
        _, T = oracle.step(g.row_ptr, g.col, g.w, t, v, 1, a_p, a_q, 0)
        assert int(C[-1]) == T, (t, v)


@pytest.mark.parametrize("pq", [(0.25, 4.0), (4.0, 0.25)])
def test_rmat_weighted_rows_equal_oracle_and_walk(pq):
    g = G.with_weights(G.rmat(13, 16, 0.57, 0.19, 0.19, 6), 2, 1, 100)
    graph = n2v.Graph.from_csr(g)
    table = n2v.StoredTable(graph, *pq)
    starts = np.arange(g.n, dtype=np.int32)
    got = n2v.stored_walk(graph, table, starts, 2, 20, 31).cpu().numpy()
    want = oracle_rows(g, starts, 20, pq[0], pq[1], 31, np.arange(g.n * 2))
    np.testing.assert_array_equal(got, want)
    fly = n2v.walk(graph, starts, 2, 20, pq[0], pq[1], 31, "persistent").cpu().numpy()
    np.testing.assert_array_equal(got, fly)


def test_er_workload_rows():
    g = G.workload_graph("er")
    graph = n2v.Graph.from_csr(g)
    table = n2v.StoredTable(graph, 0.5, 2.0)
    starts = np.arange(g.n, dtype=np.int32)
    got = n2v.stored_walk(graph, table, starts, 10, 80, 1)
    fly = n2v.walk(graph, starts, 10, 80, 0.5, 2.0, 1, "persistent")
    assert torch.equal(got, fly)
    ids = np.arange(0, g.n * 10, 37)
    np.testing.assert_array_equal(got.cpu().numpy()[ids], oracle_rows(g, starts, 80, 0.5, 2.0, 1, ids))
    # a walk-id range gives the same rows as the whole job
    part = n2v.stored_walk(graph, table, starts, 10, 80, 1, walk_begin=12345, walk_count=5000)
    assert torch.equal(part, got[12345:17345])


def test_table_is_tied_to_its_graph_and_size_checked():
    g = SMALL["und7"]
    graph = n2v.Graph.from_csr(g)
    other = n2v.Graph.from_csr(g)
    table = n2v.StoredTable(graph, 1.0, 1.0)
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    out = torch.empty((g.n, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(n2v.N2VError):
        n2v.n2v_stored_walk(other.handle, table.buf, starts, g.n, 1, 5, 1, 0, g.n, out)
    small = torch.empty(8, dtype=torch.int64, device="cuda")
    with pytest.raises(n2v.N2VError):
        n2v.n2v_stored_build(graph.handle, 1.0, 1.0, small)
    bad = torch.tensor([0, g.n], dtype=torch.int32, device="cuda")
    n2v.n2v_stored_walk(graph.handle, table.buf, bad, 2, 1, 5, 1, 0, 2, out)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_ERR_INVALID_ARG
    np.testing.assert_array_equal(out[1].cpu().numpy(), -1)
