"""CPU oracle for node2vec 2nd-order walks -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA sampler in
``paper_1805_00280_gb300``) never imports it, and the two share no code.

The C library (``n2v_oracle.c``) restates the walk model of Section 2.1 and
Section 3.2 / Algorithm 1 of the paper under the integer contract documented
in ``n2v_oracle.h``.  This module only marshals numpy arrays into it and
spreads disjoint walk-id ranges over host threads (ctypes releases the GIL
during each call, so the threads run in parallel; each walk is still computed
by the same single-threaded routine).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "n2v_oracle.c")
HDR = os.path.join(HERE, "n2v_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(verbose: bool = False) -> str:
    """Compile liboracle.so with gcc (rebuilt when the sources or the host arch change)."""
    # no contraction of a*b+c: the FN-Approx decision is made in plain IEEE double
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB, "-lm"]
    h = hashlib.sha256(" ".join(cmd).encode() + platform.machine().encode())
    for p in (SRC, HDR):
        with open(p, "rb") as f:
            h.update(f.read())
    digest = h.hexdigest()
    stamp = LIB + ".stamp"
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return LIB
    if verbose:
        print(" ".join(cmd))
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout)
    with open(stamp, "w") as f:
        f.write(digest + "\n")
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, u32, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.c_uint64)
        L.n2v_oracle_philox4x32_10.argtypes = [vp, vp, vp]
        L.n2v_oracle_philox4x32_10.restype = None
        L.n2v_oracle_draw.argtypes = [u64, u64, u32]
        L.n2v_oracle_draw.restype = u64
        L.n2v_oracle_alpha_q16.argtypes = [ctypes.c_double, ctypes.c_double, vp, vp]
        L.n2v_oracle_alpha_q16.restype = ctypes.c_int
        L.n2v_oracle_step.argtypes = [vp, vp, vp, i64, i64, i32, u32, u32, u64, vp]
        L.n2v_oracle_step.restype = i64
        L.n2v_oracle_walk.argtypes = [vp, vp, vp, vp, i64, i32, u32, u32, u64, vp, i64, vp]
        L.n2v_oracle_walk.restype = None
        L.n2v_oracle_traffic.argtypes = [vp, ctypes.c_int, vp, i64, vp, i64, vp, i32, vp]
        L.n2v_oracle_traffic.restype = None
        L.n2v_oracle_approx_decide.argtypes = [i64, i64, u32, u32, u32, u32, ctypes.c_double, vp]
        L.n2v_oracle_approx_decide.restype = ctypes.c_int
        L.n2v_oracle_walk_approx.argtypes = [vp, vp, vp, vp, i64, i32, u32, u32, u64, vp, i64, ctypes.c_double,
                                             i64, u32, u32, vp, vp]
        L.n2v_oracle_walk_approx.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _csr(row_ptr, col, w):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
    return row_ptr, col, w


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().n2v_oracle_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def draw(seed: int, walk_id: int, k: int) -> int:
    return int(lib().n2v_oracle_draw(seed, walk_id, k))


def alpha_q16(p: float, q: float) -> tuple[int, int]:
    ap, aq = ctypes.c_uint32(), ctypes.c_uint32()
    if lib().n2v_oracle_alpha_q16(p, q, ctypes.byref(ap), ctypes.byref(aq)) != 0:
        raise ValueError(f"invalid return parameters p={p} q={q}")
    return ap.value, aq.value


def step(row_ptr, col, w, t: int, v: int, k: int, a_p: int, a_q: int, u: int) -> tuple[int, int]:
    """(chosen CSR index within N(v) or -1, total T) for one step with draw u."""
    row_ptr, col, w = _csr(row_ptr, col, w)
    T = ctypes.c_uint64()
    j = lib().n2v_oracle_step(row_ptr.ctypes.data, col.ctypes.data, _ptr(w), t, v, k, a_p, a_q, u,
                              ctypes.byref(T))
    return int(j), int(T.value)


def walk(row_ptr, col, w, starts, l: int, p: float, q: float, seed: int, walk_ids,
         threads: int = 1, alpha: tuple[int, int] | None = None) -> np.ndarray:
    """Rows [len(walk_ids), l] int32 for the given walk ids (id -> starts[id mod len(starts)])."""
    row_ptr, col, w = _csr(row_ptr, col, w)
    starts = np.ascontiguousarray(starts, dtype=np.int32)
    ids = np.ascontiguousarray(walk_ids, dtype=np.int64)
    a_p, a_q = alpha if alpha is not None else alpha_q16(p, q)
    out = np.empty((ids.shape[0], l), dtype=np.int32)
    if ids.shape[0] == 0:
        return out
    L = lib()

    def run(lo: int, hi: int) -> None:
        L.n2v_oracle_walk(row_ptr.ctypes.data, col.ctypes.data, _ptr(w), starts.ctypes.data,
                          starts.shape[0], l, a_p, a_q, seed, ids[lo:].ctypes.data, hi - lo,
                          out[lo:].ctypes.data)

    threads = max(1, int(threads))
    if threads == 1:
        run(0, ids.shape[0])
    else:
        # interleaved chunks so that slow (hub-heavy) walks spread over threads
        chunk = max(1, min(1024, ids.shape[0] // (threads * 8) or 1))
        bounds = [(lo, min(lo + chunk, ids.shape[0])) for lo in range(0, ids.shape[0], chunk)]
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda b: run(*b), bounds))
    return out


def traffic(row_ptr, weighted: bool, starts, walk_ids, walks) -> tuple[int, int, int]:
    """(real transitions, model adjacency bytes, lower-model bytes) over the given rows."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    starts = np.ascontiguousarray(starts, dtype=np.int32)
    ids = np.ascontiguousarray(walk_ids, dtype=np.int64)
    walks = np.ascontiguousarray(walks, dtype=np.int32)
    out = np.zeros(3, dtype=np.uint64)
    lib().n2v_oracle_traffic(row_ptr.ctypes.data, int(weighted), starts.ctypes.data, starts.shape[0],
                             ids.ctypes.data, ids.shape[0], walks.ctypes.data, walks.shape[1],
                             out.ctypes.data)
    return int(out[0]), int(out[1]), int(out[2])


def approx_decide(deg_v: int, deg_t: int, a_p: int, a_q: int, w_min: int, w_max: int,
                  eps: float) -> tuple[bool, float, float]:
    """(approximate?, LB, UB) of FN-Approx for one step."""
    b = np.zeros(2, dtype=np.float64)
    d = lib().n2v_oracle_approx_decide(deg_v, deg_t, a_p, a_q, w_min, w_max, eps, b.ctypes.data)
    return bool(d), float(b[0]), float(b[1])


def walk_approx(row_ptr, col, w, starts, l: int, p: float, q: float, seed: int, walk_ids, eps: float,
                popular: int, threads: int = 1) -> tuple[np.ndarray, int, int]:
    """FN-Approx walks: (rows, approximated steps, 2nd-order steps).  w_min/w_max are the graph's."""
    row_ptr, col, w = _csr(row_ptr, col, w)
    starts = np.ascontiguousarray(starts, dtype=np.int32)
    ids = np.ascontiguousarray(walk_ids, dtype=np.int64)
    a_p, a_q = alpha_q16(p, q)
    w_min = int(w.min()) if w is not None and w.size else 1
    w_max = int(w.max()) if w is not None and w.size else 1
    out = np.empty((ids.shape[0], l), dtype=np.int32)
    counts = np.zeros((max(1, threads), 2), dtype=np.uint64)
    L = lib()

    def run(k: int, lo: int, hi: int) -> None:
        L.n2v_oracle_walk_approx(row_ptr.ctypes.data, col.ctypes.data, _ptr(w), starts.ctypes.data, starts.shape[0],
                                 l, a_p, a_q, seed, ids[lo:].ctypes.data, hi - lo, eps, popular, w_min, w_max,
                                 out[lo:].ctypes.data, counts[k].ctypes.data)

    if ids.shape[0]:
        bounds = np.linspace(0, ids.shape[0], max(1, threads) + 1).astype(int)
        with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
            list(ex.map(lambda k: run(k, bounds[k], bounds[k + 1]), range(max(1, threads))))
    tot = counts.sum(axis=0)
    return out, int(tot[0]), int(tot[1])
