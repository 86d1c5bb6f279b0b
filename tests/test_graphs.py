"""The seeded input generators produce canonical CSR graphs (no GPU)."""
import numpy as np
import pytest

from paper_1805_00280_gb300 import graphs as G


def check_canonical(g, symmetric=True, self_loops=False):
    rp, col = g.row_ptr, g.col
    assert rp[0] == 0 and rp[-1] == g.nnz
    assert (np.diff(rp) >= 0).all()
    assert col.min(initial=0) >= 0 and col.max(initial=0) < g.n
    src = np.repeat(np.arange(g.n), np.diff(rp))
    # strictly increasing inside each row
    same_row = src[1:] == src[:-1]
    assert (col[1:][same_row] > col[:-1][same_row]).all()
    if not self_loops:
        assert (src != col).all()
    if symmetric:
        fwd = src.astype(np.int64) * g.n + col
        bwd = col.astype(np.int64) * g.n + src
        assert np.array_equal(np.sort(fwd), np.sort(bwd))


def test_er_exact_edge_count():
    g = G.er(10_000, 100_000, 1)
    assert g.n == 10_000 and g.nnz == 200_000
    check_canonical(g)


def test_er_deterministic():
    a, b = G.er(500, 3000, 9), G.er(500, 3000, 9)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.row_ptr, b.row_ptr)
    c = G.er(500, 3000, 10)
    assert not np.array_equal(a.col, c.col)


def test_rmat_canonical_and_thread_independent():
    a = G.rmat(14, 16, 0.57, 0.19, 0.19, 1, threads=1)
    b = G.rmat(14, 16, 0.57, 0.19, 0.19, 1, threads=6)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    check_canonical(a)
    deg = a.degrees()
    # skewed: vertex 0 (all-zero id bits, quadrant a) is the largest hub
    assert deg.argmax() == 0 and deg.max() > 50 * deg.mean()


def test_rmat_uniform_parameters_are_not_skewed():
    g = G.rmat(14, 10, 0.25, 0.25, 0.25, 1)
    check_canonical(g)
    deg = g.degrees()
    assert deg.max() < 4 * deg.mean()


def test_weights_symmetric_in_range():
    g = G.with_weights(G.rmat(12, 8, 0.57, 0.19, 0.19, 2), 5, 1, 100)
    assert g.w.min() >= 1 and g.w.max() <= 100
    src = np.repeat(np.arange(g.n), g.degrees())
    key_f = src.astype(np.int64) * g.n + g.col
    key_b = g.col.astype(np.int64) * g.n + src
    of, ob = np.argsort(key_f), np.argsort(key_b)
    assert np.array_equal(g.w[of], g.w[ob])
    assert len(np.unique(g.w)) > 90


def test_uniform_streams():
    a = G.uniform(1, 0, 1000, 10_000)
    assert a.min() >= 0 and a.max() < 1000
    assert np.array_equal(a, G.uniform(1, 0, 1000, 10_000))
    assert not np.array_equal(a, G.uniform(1, 1, 1000, 10_000))


def test_from_edges_rejects_conflicts():
    with pytest.raises(ValueError):
        G.from_edges(3, [(0, 1), (1, 0)], weights=[1, 2])


def test_skew_and_wec_parameters():
    """Skew-S (Section 5.1): b = c = 0.25 and d = S a; WeC-K is (.18, .25, .25, .32)."""
    for S in (1, 2, 3, 4, 5):
        a, b, c = G.skew_abc(S)
        d = 1.0 - a - b - c
        assert b == c == 0.25 and abs(d - S * a) < 1e-12
        w = G.WORKLOADS[f"skew{S}"]
        assert w.graph["scale"] == 22 and w.r == 1 and w.l == 80 and w.pq == [(0.5, 2.0)]
    assert G.SWEEPS["skew"] == [f"skew{S}" for S in (1, 2, 3, 4, 5)]
    for K in G.SWEEPS["wec"]:
        a, b, c = G.WORKLOADS[K].graph["abc"]
        assert (a, b, c) == (0.18, 0.25, 0.25) and abs(1 - a - b - c - 0.32) < 1e-12
    # more skew puts more of the edges on fewer vertices
    lo = G.make_graph(dict(kind="rmat", scale=12, ef=50, seed=1, abc=G.skew_abc(1)))
    hi = G.make_graph(dict(kind="rmat", scale=12, ef=50, seed=1, abc=G.skew_abc(5)))
    assert hi.degrees().max() > 4 * lo.degrees().max()
