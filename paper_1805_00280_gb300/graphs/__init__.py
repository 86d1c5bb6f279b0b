"""Seeded synthetic inputs for the node2vec walk workloads (input recipe only).

The five workloads follow the shapes of the paper's evaluation (Section 4.1,
Table 1): an Erdos-Renyi graph and R-MAT graphs with the skewed (a, b, c, d)
used for power-law social networks.  Every graph is a canonical CSR: int64
``row_ptr[n+1]``, strictly increasing int32 ``col`` per row, symmetric, no
self-loops, optional symmetric uint32 weights.

Nothing here performs walk arithmetic; the generators draw from SplitMix64,
not from the Philox stream that the walks use.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from .. import _build

_LIB = None


def _lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        path = _build.build_gen()
        lib = ctypes.CDLL(path)
        i64, u64, i32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_void_p)
        lib.n2v_gen_er.argtypes = [i64, i64, u64, vp, vp]
        lib.n2v_gen_er.restype = i64
        lib.n2v_gen_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, vp, vp, i64]
        lib.n2v_gen_rmat.restype = i64
        lib.n2v_gen_weights.argtypes = [i64, vp, vp, u64, ctypes.c_uint32, ctypes.c_uint32, i32, vp]
        lib.n2v_gen_weights.restype = i32
        lib.n2v_gen_uniform.argtypes = [u64, u64, u64, i64, vp]
        lib.n2v_gen_uniform.restype = None
        lib.n2v_gen_raw64.argtypes = [u64, u64, i64, vp]
        lib.n2v_gen_raw64.restype = None
        _LIB = lib
    return _LIB


def _threads(threads: int | None) -> int:
    return int(threads or os.cpu_count() or 1)


@dataclass
class CSR:
    """A host CSR graph: ``row_ptr`` int64 [n+1], ``col`` int32 [nnz], ``w`` uint32 [nnz] or None."""

    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray | None = None
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def weighted(self) -> bool:
        return self.w is not None

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def er(n: int, m: int, seed: int) -> CSR:
    """Erdos-Renyi G(n, m): m distinct unordered pairs, no self-loops, symmetric CSR."""
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(2 * m, 1), dtype=np.int32)
    nnz = _lib().n2v_gen_er(n, m, seed, row_ptr.ctypes.data, col.ctypes.data)
    if nnz < 0:
        raise ValueError(f"n2v_gen_er failed ({nnz})")
    return CSR(row_ptr, col[:nnz], None, f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         threads: int | None = None) -> CSR:
    """R-MAT on 2^scale vertices, edge_factor * 2^scale draws, symmetrised and deduplicated."""
    n = 1 << scale
    cap = 2 * edge_factor * n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(cap, 1), dtype=np.int32)
    nnz = _lib().n2v_gen_rmat(scale, edge_factor, a, b, c, seed, _threads(threads),
                              row_ptr.ctypes.data, col.ctypes.data, cap)
    if nnz < 0:
        raise ValueError(f"n2v_gen_rmat failed ({nnz})")
    return CSR(row_ptr, col[:nnz], None, f"rmat{scale}_ef{edge_factor}_s{seed}")


def with_weights(g: CSR, seed: int, lo: int = 1, hi: int = 100, threads: int | None = None) -> CSR:
    """Attach symmetric weights uniform in [lo, hi]: w(u,v) == w(v,u)."""
    w = np.empty(max(g.nnz, 1), dtype=np.uint32)
    rc = _lib().n2v_gen_weights(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data, seed, lo, hi,
                                _threads(threads), w.ctypes.data)
    if rc != 0:
        raise ValueError("n2v_gen_weights failed")
    return CSR(g.row_ptr, g.col, w[: g.nnz], g.name + f"_w{lo}-{hi}")


def uniform(seed: int, stream: int, n: int, count: int) -> np.ndarray:
    """``count`` integers uniform in [0, n) from the SplitMix64 stream (seed, stream)."""
    out = np.empty(max(count, 1), dtype=np.int64)
    _lib().n2v_gen_uniform(seed, stream, n, count, out.ctypes.data)
    return out[:count]


def raw64(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.uint64)
    _lib().n2v_gen_raw64(seed, stream, count, out.ctypes.data)
    return out[:count]


def from_edges(n: int, edges, weights=None, symmetric: bool = True) -> CSR:
    """Small hand-made graphs for tests: canonical CSR from an edge list.

    With ``symmetric`` each (u, v) also adds (v, u).  Duplicates are rejected
    so that the result is canonical; weights follow their edge.
    """
    adj: dict[int, dict[int, int]] = {u: {} for u in range(n)}
    for i, (u, v) in enumerate(edges):
        wt = 1 if weights is None else int(weights[i])
        pairs = [(u, v), (v, u)] if symmetric and u != v else [(u, v)]
        for a, b in pairs:
            if b in adj[a] and adj[a][b] != wt:
                raise ValueError("conflicting duplicate edge")
            adj[a][b] = wt
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for u in range(n):
        nb = sorted(adj[u])
        row_ptr[u + 1] = row_ptr[u] + len(nb)
        cols += nb
        ws += [adj[u][x] for x in nb]
    w = None if weights is None else np.asarray(ws, dtype=np.uint32)
    return CSR(row_ptr, np.asarray(cols, dtype=np.int32), w, "edges")


# --------------------------------------------------------------------------
# The five workloads.

RMAT_SOCIAL = (0.57, 0.19, 0.19)  # d = 0.05


@dataclass
class Workload:
    name: str
    graph: dict
    r: int
    l: int
    pq: list = field(default_factory=list)
    seed: int = 1
    note: str = ""


WORKLOADS = {
    "er": Workload("er", dict(kind="er", n=10_000, m=100_000, seed=1), r=10, l=80, pq=[(0.5, 2.0)],
                   note="ER G(n=1e4, m=1e5), r=10, l=80, p=0.5, q=2"),
    "rmat20": Workload("rmat20", dict(kind="rmat", scale=20, ef=16, seed=1), r=10, l=80,
                       pq=[(1.0, 1.0), (0.25, 4.0), (4.0, 0.25)],
                       note="R-MAT scale 20, ef 16, (.57,.19,.19,.05), r=10, l=80"),
    "rmat23w": Workload("rmat23w", dict(kind="rmat", scale=23, ef=16, seed=1, weights=(1, 100)), r=4,
                        l=80, pq=[(1.0, 0.5)],
                        note="weighted R-MAT scale 23, ef 16, w in [1,100], r=4, l=80, p=1, q=0.5"),
    "rmat26": Workload("rmat26", dict(kind="rmat", scale=26, ef=16, seed=1), r=1, l=80, pq=[(2.0, 0.5)],
                       note="R-MAT scale 26, ef 16, r=1, l=80, p=2, q=0.5"),
    # the scale-26 walk parameters on a graph whose col array (0.5 GB) still exceeds L2: the case
    # small enough for a full ncu capture of one launch
    "rmat22": Workload("rmat22", dict(kind="rmat", scale=22, ef=16, seed=1), r=1, l=80, pq=[(2.0, 0.5)],
                       note="R-MAT scale 22, ef 16, r=1, l=80, p=2, q=0.5"),
    "rmat24serve": Workload("rmat24serve", dict(kind="rmat", scale=24, ef=16, seed=1), r=1, l=80,
                            pq=[], note="serving on R-MAT scale 24, ef 16"),
    # skewed but small enough for a stored transition table (8 sum d^2 = 76 GB)
    "rmat18": Workload("rmat18", dict(kind="rmat", scale=18, ef=16, seed=1), r=10, l=80,
                       pq=[(1.0, 1.0), (0.25, 4.0), (4.0, 0.25)],
                       note="R-MAT scale 18, ef 16, (.57,.19,.19,.05), r=10, l=80"),
}


def skew_abc(S: float) -> tuple[float, float, float]:
    """R-MAT (a, b, c) of the Skew-S graphs (Section 5.1): b = c = 0.25 and d = S a."""
    a = 0.5 / (1.0 + S)
    return (a, 0.25, 0.25)


# Skew-S: 2^22 vertices, average degree about 100 (50 generated edges per vertex,
# symmetrised), one walk of length 80 per vertex at p = 0.5, q = 2 (Section 5.1)
for _S in (1, 2, 3, 4, 5):
    WORKLOADS[f"skew{_S}"] = Workload(f"skew{_S}", dict(kind="rmat", scale=22, ef=50, seed=1, abc=skew_abc(_S)),
                                      r=1, l=80, pq=[(0.5, 2.0)],
                                      note=f"Skew-{_S}: R-MAT scale 22, ef 50, d = {_S} a, b = c = 0.25, r=1, l=80")
# WeC-K: 2^K vertices, about 100 x 2^K adjacency entries, (a, b, c, d) = (.18, .25, .25, .32)
for _K in (20, 21, 22, 23):
    WORKLOADS[f"wec{_K}"] = Workload(f"wec{_K}", dict(kind="rmat", scale=_K, ef=50, seed=1, abc=(0.18, 0.25, 0.25)),
                                     r=1, l=80, pq=[(0.5, 2.0)],
                                     note=f"WeC-{_K}: R-MAT scale {_K}, ef 50, (.18,.25,.25,.32), r=1, l=80")

SWEEPS = {"skew": [f"skew{S}" for S in (1, 2, 3, 4, 5)], "wec": [f"wec{K}" for K in (20, 21, 22, 23)]}


def make_graph(spec: dict, threads: int | None = None) -> CSR:
    if spec["kind"] == "er":
        g = er(spec["n"], spec["m"], spec["seed"])
    elif spec["kind"] == "rmat":
        a, b, c = spec.get("abc", RMAT_SOCIAL)
        g = rmat(spec["scale"], spec["ef"], a, b, c, spec["seed"], threads)
    else:
        raise ValueError(spec)
    if spec.get("weights"):
        lo, hi = spec["weights"]
        g = with_weights(g, spec["seed"] + 1000, lo, hi, threads)
    return g


def workload_graph(name: str, threads: int | None = None) -> CSR:
    return make_graph(WORKLOADS[name].graph, threads)
