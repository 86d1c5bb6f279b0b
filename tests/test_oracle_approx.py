"""Pins for FN-Approx in the oracle (Section 3.4, Eq. 2-3), no GPU.

* The bounds bracket the exact transition probabilities: on random undirected
  graphs, every exact P(v -> x), x != t, computed with rational arithmetic from
  the model's definition, lies in [LB, UB] (the paper's claim for Eq. 2-3).
* The double-precision decision UB - LB < eps agrees with the same comparison
  in exact rational arithmetic wherever the two are not within rounding of eps.
* eps = 0 reproduces the exact walks; an approximated step samples by static
  weights (chi-squared against the static distribution at a hub).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1805_00280_gb300 import graphs as G

scipy_stats = pytest.importorskip("scipy.stats")


def exact_bounds(dv, dt, a_p, a_q, w_min, w_max):
    ip, iq = Fraction(a_p, 65536), Fraction(a_q, 65536)
    others, cmax = dv - 1, min(dt, dv - 1)
    num_min = w_min * min(iq, Fraction(1))
    num_max = w_max * max(iq, Fraction(1))
    all_q = ip + others * iq
    most_1 = ip + cmax + (others - cmax) * iq
    den_min = w_min * (most_1 if iq >= 1 else all_q)
    den_max = w_max * (all_q if iq >= 1 else most_1)
    return num_min / den_max, num_max / den_min


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("pq", [(1.0, 1.0), (0.5, 2.0), (2.0, 0.5), (0.25, 4.0), (4.0, 0.25)])
def test_bounds_bracket_exact_probabilities(weighted, pq):
    g = G.rmat(9, 8, 0.57, 0.19, 0.19, 13)
    if weighted:
        g = G.with_weights(g, 3, 1, 9)
    w = g.w if g.w is not None else np.ones(g.nnz, dtype=np.uint32)
    w_min, w_max = int(w.min()), int(w.max())
    a_p, a_q = oracle.alpha_q16(*pq)
    rng = np.random.default_rng(1)
    src = np.repeat(np.arange(g.n), g.degrees())
    checked = 0
    for e in rng.choice(g.nnz, 150, replace=False):
        t, v = int(src[e]), int(g.col[e])
        nt = set(g.col[g.row_ptr[t]:g.row_ptr[t + 1]].tolist())
        b, end = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        cs = []
        for j in range(b, end):
            x = int(g.col[j])
            a = a_p if x == t else (65536 if x in nt else a_q)
            cs.append((x, int(w[j]) * a))
        T = sum(c for _, c in cs)
        _, lb, ub = oracle.approx_decide(end - b, len(nt), a_p, a_q, w_min, w_max, 1e-3)
        elb, eub = exact_bounds(end - b, len(nt), a_p, a_q, w_min, w_max)
        assert abs(lb - float(elb)) <= 1e-15 * max(1.0, float(elb)) * 4
        assert abs(ub - float(eub)) <= 1e-15 * max(1.0, float(eub)) * 4
        for x, c in cs:
            if x == t:
                continue
            prob = Fraction(c, T)
            assert elb <= prob <= eub, (t, v, x)
            checked += 1
    assert checked > 100


def test_decision_matches_exact_rational():
    rng = np.random.default_rng(7)
    agree = 0
    for _ in range(3000):
        dv = int(rng.integers(2, 200_000))
        dt = int(rng.integers(1, 5000))
        a_p = int(rng.integers(1, 1 << 20))
        a_q = int(rng.integers(1, 1 << 20))
        w_min = int(rng.integers(1, 50))
        w_max = w_min + int(rng.integers(0, 50))
        eps = float(10 ** rng.uniform(-6, -1))
        d, _, _ = oracle.approx_decide(dv, dt, a_p, a_q, w_min, w_max, eps)
        elb, eub = exact_bounds(dv, dt, a_p, a_q, w_min, w_max)
        gap = eub - elb
        if abs(float(gap) - eps) <= 1e-9 * eps:
            continue  # within rounding of the threshold: either branch is a faithful rounding
        assert d == (gap < Fraction(eps))
        agree += 1
    assert agree > 2900


def test_eps_zero_is_exact():
    g = G.rmat(12, 16, 0.57, 0.19, 0.19, 2)
    starts = np.arange(g.n, dtype=np.int32)
    ids = np.arange(0, g.n, 3)
    exact = oracle.walk(g.row_ptr, g.col, None, starts, 20, 0.5, 2.0, 4, ids)
    rows, n_approx, n2 = oracle.walk_approx(g.row_ptr, g.col, None, starts, 20, 0.5, 2.0, 4, ids, 0.0, 8)
    assert n_approx == 0 and n2 > 0
    np.testing.assert_array_equal(rows, exact)


def test_approximated_hub_steps_follow_static_weights():
    # leaf -> hub -> ?  with the hub popular and the leaf not: approximated, so
    # the next vertex is uniform over the hub's 4000 leaves (static weights),
    # including the leaf it came from (exact node2vec would favour it by 1/p)
    m = 4000
    star = G.from_edges(m + 1, [(0, i) for i in range(1, m + 1)])
    rows, n_approx, n2 = oracle.walk_approx(star.row_ptr, star.col, None, np.array([1], np.int32), 2, 0.25, 1.0, 5,
                                            np.arange(400_000), 1e-3, 100, threads=4)
    assert n_approx == n2 == 400_000
    back = float(np.mean(rows[:, 1] == 1))
    assert abs(back - 1 / m) < 5 * np.sqrt((1 / m) * (1 - 1 / m) / 400_000)
    counts = np.bincount(rows[:, 1], minlength=m + 1)[1:]
    assert scipy_stats.chisquare(counts).pvalue > 1e-3
    # the exact walk returns with probability a_p / (a_p + (m - 1) a_q), about 4x more
    exact = oracle.walk(star.row_ptr, star.col, None, np.array([1], np.int32), 2, 0.25, 1.0, 5, np.arange(400_000))
    assert float(np.mean(exact[:, 1] == 1)) > 3 * back


def test_approximation_triggers_on_rmat():
    g = G.rmat(13, 16, 0.57, 0.19, 0.19, 2)
    starts = np.arange(g.n, dtype=np.int32)
    rows, n_approx, n2 = oracle.walk_approx(g.row_ptr, g.col, None, starts, 40, 1.0, 1.0, 4, np.arange(g.n), 1e-2,
                                            256, threads=4)
    assert 0 < n_approx < n2
    # the rows still follow edges
    adj = set(zip(np.repeat(np.arange(g.n), g.degrees()).tolist(), g.col.tolist()))
    for s0, row in zip(starts[:500], rows[:500]):
        prev = int(s0)
        for x in row.tolist():
            if x < 0:
                break
            assert (prev, x) in adj
            prev = x


def test_popular_threshold_is_strict_for_t():
    """A step is approximated only when deg(v) >= popular and deg(t) < popular."""
    m, extra = 3000, 9
    # hub 0 joined to leaves 1..m; leaf 1 also joined to m+1..m+extra: deg(1) = 1 + extra
    edges = [(0, i) for i in range(1, m + 1)] + [(1, m + j) for j in range(1, extra + 1)]
    g = G.from_edges(m + extra + 1, edges)
    deg1 = int(g.degrees()[1])
    ids = np.arange(20_000)
    _, n_at, _ = oracle.walk_approx(g.row_ptr, g.col, None, np.array([1], np.int32), 2, 0.5, 2.0, 3, ids, 1e-2,
                                    deg1)
    _, n_above, _ = oracle.walk_approx(g.row_ptr, g.col, None, np.array([1], np.int32), 2, 0.5, 2.0, 3, ids, 1e-2,
                                       deg1 + 1)
    assert n_at == 0  # deg(t) == popular: t is popular, no approximation
    assert n_above > 0  # deg(t) < popular and the hub has deg >= popular
