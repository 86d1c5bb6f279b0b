"""Small hand-built graphs shared by the oracle pins and the GPU parity tests."""
import numpy as np

from paper_1805_00280_gb300 import graphs as G


def small_graphs():
    rng = np.random.default_rng(2024)
    out = {}
    # a 7-vertex undirected graph with triangles, a pendant vertex and a square
    e1 = [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5), (5, 6), (6, 3), (2, 5), (0, 6)]
    out["und7"] = G.from_edges(7, e1)
    out["und7w"] = G.from_edges(7, e1, weights=list(rng.integers(1, 10, len(e1))))
    # K5 with weights (every non-return neighbour is a common neighbour)
    k5 = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    out["k5w"] = G.from_edges(5, k5, weights=list(rng.integers(1, 6, len(k5))))
    # directed, with a sink (vertex 5), a self-loop at 1 and an asymmetric pair
    d = [(0, 1), (1, 1), (1, 2), (2, 0), (2, 3), (3, 1), (3, 4), (4, 2), (4, 5), (0, 3), (1, 4)]
    out["dir6"] = G.from_edges(6, d, symmetric=False)
    # directed weighted with a zero-weight edge (never chosen)
    dw = [(0, 1), (1, 0), (1, 2), (2, 1), (2, 0), (0, 2), (2, 3), (3, 2), (1, 3)]
    out["dir4w0"] = G.from_edges(4, dw, weights=[3, 1, 0, 2, 5, 1, 4, 2, 1], symmetric=False)
    # random graph on 8 vertices
    pairs = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    pick = rng.choice(len(pairs), 14, replace=False)
    out["rand8"] = G.from_edges(8, [pairs[i] for i in sorted(pick)])
    return out


def big_star(leaves: int):
    """Hub 0 joined to `leaves` leaves: a step at the hub sees deg(v) = leaves, deg(t) = 1."""
    rp = np.zeros(leaves + 2, dtype=np.int64)
    rp[1] = leaves
    rp[2:] = leaves + np.arange(1, leaves + 1)
    col = np.concatenate([np.arange(1, leaves + 1, dtype=np.int32), np.zeros(leaves, dtype=np.int32)])
    return G.CSR(rp, col, None, f"star{leaves}")


def two_hubs(m: int, extra: int = 0):
    """K_{2,m} plus the hub-hub edge and `extra` pendant chains: both endpoints of
    a hub-to-hub step have ~m neighbours, almost all of them common."""
    edges = [(0, 1)] + [(h, 2 + i) for h in (0, 1) for i in range(m)]
    edges += [(2 + i, 2 + m + i) for i in range(extra)]
    return G.from_edges(2 + m + extra, edges)
