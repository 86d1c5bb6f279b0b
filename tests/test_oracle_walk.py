"""Pins for the CPU oracle's walks against what the paper and mathematics fix (no GPU).

The paper prints no walk or numeric example, so the oracle is pinned by:

* exact path enumeration on graphs of <= 8 vertices (rational probabilities
  from the definition in Section 2.1: alpha = 1/p for x == t, 1 for x in
  N(t), 1/q otherwise; first step by static weights, Algorithm 1 superstep 0)
  against the frequencies of 10^6 oracle walks, by a chi-squared test;
* closed forms for the probability of returning to t on K_n, C_n, stars and
  complete bipartite graphs, by a binomial z-test;
* the p = q = 1 case, which must reproduce a textbook first-order
  inverse-CDF walk (numpy cumsum + searchsorted) draw for draw;
* exact selection boundaries of the scaled draw r = floor(u T / 2^64);
* invariants: every step follows an edge, dead ends pad with -1;
* the paper's qualitative claims: low p favours returning, walks visit
  high-degree vertices more often (Section 2.1, Section 3.3).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1805_00280_gb300 import graphs as G
from small_graphs import small_graphs

scipy_stats = pytest.importorskip("scipy.stats")


# --------------------------------------------------------------------------
# helpers (independent of the oracle's code)

def adjacency(g):
    rp, col = g.row_ptr, g.col
    w = g.w if g.w is not None else np.ones(g.nnz, dtype=np.uint32)
    return [[(int(col[e]), int(w[e])) for e in range(rp[u], rp[u + 1])] for u in range(g.n)]


def path_distribution(g, s0, l, a_p, a_1, a_q):
    """Exact probability of every length-l row from start s0 (rows padded with -1)."""
    adj = adjacency(g)
    nbset = [set(x for x, _ in a) for a in adj]
    out = {}

    def rec(path, t, v, k, prob):
        if k == l:
            out[tuple(path)] = out.get(tuple(path), 0) + prob
            return
        cs = []
        for x, wt in adj[v]:
            if k == 0:
                a = 1
            elif x == t:
                a = a_p
            elif x in nbset[t]:
                a = a_1
            else:
                a = a_q
            cs.append(wt * a)
        T = sum(cs)
        if T == 0:
            key = tuple(path + [-1] * (l - k))
            out[key] = out.get(key, 0) + prob
            return
        for (x, _), c in zip(adj[v], cs):
            if c:
                rec(path + [x], v, x, k + 1, prob * Fraction(c) / Fraction(T))

    rec([], -1, s0, 0, Fraction(1))
    return out


def chi2_pvalue(rows, dist):
    n = rows.shape[0]
    keys, counts = np.unique(rows, axis=0, return_counts=True)
    observed = {tuple(int(x) for x in k): int(c) for k, c in zip(keys, counts)}
    impossible = [k for k in observed if k not in dist]
    assert not impossible, f"oracle produced impossible rows {impossible[:3]}"
    exp, obs = [], []
    rest_e, rest_o = 0.0, 0
    for k, pr in dist.items():
        e = float(pr) * n
        o = observed.get(k, 0)
        if e < 5:
            rest_e += e
            rest_o += o
        else:
            exp.append(e)
            obs.append(o)
    if rest_e > 0:
        exp.append(rest_e)
        obs.append(rest_o)
    exp, obs = np.array(exp), np.array(obs)
    if len(exp) < 2:
        return 1.0
    stat = float(((obs - exp) ** 2 / exp).sum())
    return float(scipy_stats.chi2.sf(stat, len(exp) - 1))


def run(g, starts, l, p, q, seed, ids, alpha=None):
    return oracle.walk(g.row_ptr, g.col, g.w, np.asarray(starts, dtype=np.int32), l, p, q, seed,
                       np.asarray(ids, dtype=np.int64), threads=4, alpha=alpha)


# --------------------------------------------------------------------------
# small graphs for enumeration

SMALL = small_graphs()
PQ = [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25), (0.5, 2.0), (3.0, 0.7)]
ENUM_CASES = [(name, s0, pq) for name, s0 in [("und7", 0), ("und7w", 3), ("k5w", 1), ("dir6", 0),
                                               ("dir4w0", 0), ("rand8", 2)] for pq in PQ]


@pytest.mark.parametrize("name,s0,pq", ENUM_CASES, ids=[f"{a}-s{b}-p{c[0]}q{c[1]}" for a, b, c in ENUM_CASES])
def test_enumeration_chi2(name, s0, pq):
    g = SMALL[name]
    p, q = pq
    l = 4
    n = 1_000_000 if name in ("und7", "dir6", "und7w") else 300_000
    a_p, a_q = oracle.alpha_q16(p, q)
    rows = run(g, [s0], l, p, q, seed=17 + len(name), ids=np.arange(n))
    dist_q16 = path_distribution(g, s0, l, a_p, 65536, a_q)
    assert sum(dist_q16.values()) == 1
    assert chi2_pvalue(rows, dist_q16) > 1e-3
    # the real-valued alpha gives the same outcome: Q16 rounding is below 2^-17 relative
    dist_real = path_distribution(g, s0, l, 1 / Fraction(p), Fraction(1), 1 / Fraction(q))
    assert chi2_pvalue(rows, dist_real) > 1e-3


def test_enumeration_catches_a_swapped_alpha():
    """The chi-squared pin has power: swapping p and q on the expected side is rejected."""
    g = SMALL["und7"]
    rows = run(g, [0], 4, 0.25, 4.0, seed=3, ids=np.arange(300_000))
    a_p, a_q = oracle.alpha_q16(0.25, 4.0)
    wrong = path_distribution(g, 0, 4, a_q, 65536, a_p)
    assert chi2_pvalue(rows, wrong) < 1e-6


# --------------------------------------------------------------------------
# closed forms: probability that the second step returns to the start

def backtrack_rate(g, s0, p, q, n=400_000, seed=5):
    rows = run(g, [s0], 2, p, q, seed, np.arange(n))
    return float(np.mean(rows[:, 1] == s0)), n


def ztest(hat, prob, n):
    prob = float(prob)
    return abs(hat - prob) / np.sqrt(prob * (1 - prob) / n)


@pytest.mark.parametrize("p,q", [(1.0, 1.0), (0.25, 4.0), (4.0, 0.25), (0.5, 2.0)])
def test_closed_forms(p, q):
    a_p, a_q = oracle.alpha_q16(p, q)
    one = 65536
    # K_n: all other neighbours of v are neighbours of t
    n = 7
    kn = G.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    hat, N = backtrack_rate(kn, 0, p, q)
    assert ztest(hat, Fraction(a_p, a_p + (n - 2) * one), N) < 4.5
    # C_n (n >= 5): the other neighbour of v is two hops from t
    cn = G.from_edges(9, [(i, (i + 1) % 9) for i in range(9)])
    hat, N = backtrack_rate(cn, 0, p, q)
    assert ztest(hat, Fraction(a_p, a_p + a_q), N) < 4.5
    # star, leaf -> hub -> : the other leaves are two hops from the leaf
    m = 6
    star = G.from_edges(m + 1, [(0, i) for i in range(1, m + 1)])
    hat, N = backtrack_rate(star, 3, p, q)
    assert ztest(hat, Fraction(a_p, a_p + (m - 1) * a_q), N) < 4.5
    # K_{a,b}: from v in B, the neighbours are the a vertices of A, none adjacent to t
    a, b = 4, 3
    kab = G.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    hat, N = backtrack_rate(kab, 0, p, q)
    assert ztest(hat, Fraction(a_p, a_p + (a - 1) * a_q), N) < 4.5


def test_closed_form_weighted_star():
    ws = [5, 1, 7, 2, 9, 3]
    star = G.from_edges(7, [(0, i) for i in range(1, 7)], weights=ws)
    a_p, a_q = oracle.alpha_q16(0.5, 2.0)
    hat, N = backtrack_rate(star, 2, 0.5, 2.0)
    w_back = ws[1]
    rest = sum(ws) - w_back
    assert ztest(hat, Fraction(w_back * a_p, w_back * a_p + rest * a_q), N) < 4.5


def test_low_p_favours_return():
    g = G.rmat(12, 8, 0.57, 0.19, 0.19, 3)
    rows_lo = run(g, np.arange(g.n), 20, 0.25, 1.0, 9, np.arange(g.n))
    rows_hi = run(g, np.arange(g.n), 20, 4.0, 1.0, 9, np.arange(g.n))

    def ret(rows):
        r = rows[:, 2:]
        back = (r == rows[:, :-2]) & (r >= 0)
        return back.sum() / max(1, (r >= 0).sum())

    assert ret(rows_lo) > 2 * ret(rows_hi)


# --------------------------------------------------------------------------
# exact selection boundaries

def test_selection_boundaries_exact():
    """u maps to index j exactly when C_{j-1} <= floor(u T / 2^64) < C_j."""
    ws = [5, 1, 7, 2, 9, 3]
    star = G.from_edges(7, [(0, i) for i in range(1, 7)], weights=ws)
    a_p, a_q = oracle.alpha_q16(0.5, 2.0)
    t, v = 2, 0  # came from leaf 2 into the hub: x=2 returns, other leaves are 2 hops away
    c = [w * (a_p if leaf == t else a_q) for leaf, w in zip(range(1, 7), ws)]
    C = np.cumsum(c).tolist()
    T = C[-1]
    j0, T0 = oracle.step(star.row_ptr, star.col, star.w, t, v, 1, a_p, a_q, 0)
    assert T0 == T and j0 == 0
    j_last, _ = oracle.step(star.row_ptr, star.col, star.w, t, v, 1, a_p, a_q, 2**64 - 1)
    assert j_last == len(c) - 1
    for j in range(1, len(c)):
        u = -(-C[j - 1] * 2**64 // T)  # smallest u with floor(u T / 2^64) >= C_{j-1}
        assert oracle.step(star.row_ptr, star.col, star.w, t, v, 1, a_p, a_q, u)[0] == j
        assert oracle.step(star.row_ptr, star.col, star.w, t, v, 1, a_p, a_q, u - 1)[0] == j - 1


def test_step_zero_ignores_t():
    g = SMALL["und7w"]
    for u in [0, 2**63, 2**64 - 1, 123456789]:
        assert oracle.step(g.row_ptr, g.col, g.w, 1, 3, 0, 1, 1, u) == \
            oracle.step(g.row_ptr, g.col, g.w, 5, 3, 0, 9, 99, u)


# --------------------------------------------------------------------------
# p = q = 1 reproduces the textbook first-order walk, draw for draw

def first_order_numpy(g, starts, l, seed, ids):
    """Inverse-CDF first-order walk: P_j = cumsum(w), r = floor(u S / 2^64), first P_j > r."""
    w = g.w if g.w is not None else np.ones(g.nnz, dtype=np.uint32)
    out = np.full((len(ids), l), -1, dtype=np.int32)
    for i, wid in enumerate(ids):
        v = int(starts[wid % len(starts)])
        for k in range(l):
            b, e = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
            P = np.cumsum(w[b:e].astype(np.uint64))
            if e == b or int(P[-1]) == 0:
                break
            u = oracle.draw(seed, int(wid), k)
            r1 = (u * int(P[-1])) >> 64
            j = int(np.searchsorted(P, np.uint64(r1), side="right"))
            v = int(g.col[b + j])
            out[i, k] = v
    return out


@pytest.mark.parametrize("weighted", [False, True])
def test_p_q_one_is_first_order(weighted):
    g = G.rmat(11, 8, 0.57, 0.19, 0.19, 5)
    if weighted:
        g = G.with_weights(g, 77, 1, 100)
    starts = np.arange(g.n, dtype=np.int32)
    ids = np.arange(0, 3 * g.n, 7)[:1500]
    got = run(g, starts, 30, 1.0, 1.0, 42, ids)
    want = first_order_numpy(g, starts, 30, 42, ids)
    np.testing.assert_array_equal(got, want)


def test_first_order_differs_when_p_q_not_one():
    g = G.rmat(11, 8, 0.57, 0.19, 0.19, 5)
    starts = np.arange(g.n, dtype=np.int32)
    ids = np.arange(0, 500)
    got = run(g, starts, 30, 0.25, 4.0, 42, ids)
    want = first_order_numpy(g, starts, 30, 42, ids)
    assert (got != want).any()


# --------------------------------------------------------------------------
# invariants

def test_every_step_follows_an_edge():
    g = G.rmat(13, 16, 0.57, 0.19, 0.19, 2)
    starts = np.arange(g.n, dtype=np.int32)
    ids = np.arange(0, 2 * g.n, 3)
    rows = run(g, starts, 40, 0.5, 2.0, 1, ids)
    adj = set(zip(np.repeat(np.arange(g.n), g.degrees()).tolist(), g.col.tolist()))
    deg = g.degrees()
    for i, wid in enumerate(ids):
        s0 = int(starts[wid % g.n])
        row = rows[i]
        if deg[s0] == 0:
            assert (row == -1).all()
            continue
        # undirected: a walk that takes one step never dead-ends
        assert (row >= 0).all()
        prev = s0
        for x in row.tolist():
            assert (prev, x) in adj
            prev = x


def test_dead_end_pads_with_minus_one():
    g = SMALL["dir6"]  # vertex 5 is a sink, reached from 4
    rows = run(g, [4], 5, 1.0, 1.0, 11, np.arange(2000))
    hit = np.where(rows[:, 0] == 5)[0]
    assert hit.size > 0
    assert (rows[hit, 1:] == -1).all()
    for r in rows:
        nz = np.where(r == -1)[0]
        if nz.size:
            assert (r[nz[0]:] == -1).all()
            assert r[nz[0] - 1] == 5 if nz[0] > 0 else True


def test_zero_weight_edges_never_chosen():
    g = SMALL["dir4w0"]  # edge 1->2 has weight 0
    rows = run(g, [0, 1, 2, 3], 6, 0.5, 2.0, 3, np.arange(40_000))
    starts = np.array([0, 1, 2, 3])
    full = np.concatenate([starts[np.arange(40_000) % 4][:, None], rows], axis=1)
    pairs = set(zip(full[:, :-1].ravel().tolist(), full[:, 1:].ravel().tolist()))
    assert (1, 2) not in pairs


def test_round_major_walk_ids():
    g = SMALL["und7"]
    starts = np.array([3, 5, 1], dtype=np.int32)
    ids = np.arange(9)
    rows = run(g, starts, 3, 0.5, 2.0, 4, ids)
    # walk id i starts at starts[i mod 3]: its first step is a neighbour of that start
    for i in ids:
        s0 = starts[i % 3]
        assert rows[i, 0] in g.col[g.row_ptr[s0]:g.row_ptr[s0 + 1]]
    # ids are the only input: the same id gives the same row wherever it sits
    again = run(g, starts, 3, 0.5, 2.0, 4, ids[::-1])
    np.testing.assert_array_equal(again[::-1], rows)


def test_visits_grow_with_degree():
    g = G.rmat(13, 16, 0.57, 0.19, 0.19, 4)
    deg = g.degrees()
    starts = np.flatnonzero(deg > 0).astype(np.int32)
    rows = run(g, starts, 40, 1.0, 1.0, 8, np.arange(starts.size))
    visits = np.bincount(rows[rows >= 0].ravel(), minlength=g.n)
    has = deg > 0
    rho = scipy_stats.spearmanr(deg[has], visits[has]).correlation
    assert rho > 0.5


def test_traffic_model_counts():
    g = SMALL["und7w"]
    starts = np.array([0, 4], dtype=np.int32)
    ids = np.arange(6)
    rows = run(g, starts, 5, 0.5, 2.0, 4, ids)
    deg = g.degrees()
    steps = bytes_ = lower = 0
    for i, wid in enumerate(ids):
        s0 = int(starts[wid % 2])
        for k in range(5):
            if rows[i, k] < 0:
                break
            v = s0 if k == 0 else int(rows[i, k - 1])
            b = 16 + 8 * int(deg[v]) + 4
            lower += b
            if k >= 1:
                t = s0 if k == 1 else int(rows[i, k - 2])
                b += 16 + 4 * int(deg[t])
            steps += 1
            bytes_ += b
    assert oracle.traffic(g.row_ptr, True, starts, ids, rows) == (steps, bytes_, lower)
