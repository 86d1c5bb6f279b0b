"""Python binding of the C ABI in include/n2v.h (argument marshalling only).

Every function named ``n2v_*`` here calls the C entry point of the same name
in the in-tree ``lib/libn2v.so``; tensors are passed as raw device pointers
and streams as ``cudaStream_t`` handles.  PyTorch only supplies device memory
and streams.  There is no CPU or PyTorch fallback: if the CUDA library is
missing, importing this module raises.

``Graph`` and ``walk`` are conveniences that allocate the caller-owned buffers
with torch and then call the same entry points.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

N2V_OK = 0
N2V_ERR_INVALID_ARG = -1
N2V_ERR_INVALID_GRAPH = -2
N2V_ERR_OVERFLOW = -3
N2V_ERR_NO_MEM = -4
N2V_ERR_TIMEOUT = -5
N2V_ERR_CUDA = -6
N2V_ERR_INTERNAL = -7

N2V_PLAIN = 0
N2V_BINNED = 1
N2V_PERSISTENT = 2
N2V_FLAG_CUDA_GRAPH = 0x100

VARIANTS = {"plain": N2V_PLAIN, "binned": N2V_BINNED, "persistent": N2V_PERSISTENT}


class N2VError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {n2v_strerror(code)} ({code})" if what else f"{n2v_strerror(code)} ({code})")


class n2v_tune(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("thread_max_deg", ctypes.c_int32), ("smem_specials", ctypes.c_int32),
                ("hub_count", ctypes.c_int32), ("hub_min_degree", ctypes.c_int32),
                ("chunk_walkers", ctypes.c_int32), ("hub_budget_mb", ctypes.c_int32),
                ("stage_window", ctypes.c_int32), ("stream_ratio", ctypes.c_int32),
                ("spill_specials", ctypes.c_int32), ("stage_buffers", ctypes.c_int32),
                ("bitmap_hubs", ctypes.c_int32), ("block_min_deg", ctypes.c_int32),
                ("merge_ratio", ctypes.c_int32), ("l2_persist_mb", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class n2v_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("weighted", ctypes.c_int32),
                ("hub_count", ctypes.c_int32), ("max_degree", ctypes.c_int64), ("max_wsum", ctypes.c_uint64),
                ("hub_min_degree", ctypes.c_int64), ("hub_slots", ctypes.c_int64),
                ("deg_hist", ctypes.c_int64 * 34), ("w_min", ctypes.c_uint32), ("w_max", ctypes.c_uint32),
                ("bitmap_hubs", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("bitmap_min_degree", ctypes.c_int64)]


class n2v_job(ctypes.Structure):
    _fields_ = [("starts", ctypes.c_void_p), ("n_starts", ctypes.c_int64), ("l", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class n2v_serve_cfg(ctypes.Structure):
    _fields_ = [("tick_walkers", ctypes.c_int64), ("max_jobs_per_tick", ctypes.c_int32),
                ("spill_specials", ctypes.c_int32), ("min_share", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class n2v_serve_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("active", ctypes.c_int64), ("arena_used", ctypes.c_int64),
                ("arena_bytes", ctypes.c_int64), ("ticks", ctypes.c_int64)]


_LIB = None


def checked() -> bool:
    """True when this process uses the checked build (environment N2V_CHECKED=1): the same
    library with device self-checks that report failures as N2V_ERR_INTERNAL."""
    return os.environ.get("N2V_CHECKED") == "1"


def stats_build() -> bool:
    """True when this process uses the stats build (environment N2V_STATS=1): the same library
    with per-kind step counters that n2v_step_stats reads."""
    return os.environ.get("N2V_STATS") == "1"


def lib() -> ctypes.CDLL:
    """Load libn2v.so, or libn2v_checked.so under N2V_CHECKED=1, or libn2v_stats.so under
    N2V_STATS=1 (building it in-tree when its sources changed)."""
    global _LIB
    if _LIB is None:
        path = _build.LIBN2V_CHECKED if checked() else (_build.LIBN2V_STATS if stats_build() else _build.LIBN2V)
        if not os.path.exists(path) or os.environ.get("N2V_NO_AUTOBUILD") != "1":
            path = _build.build_n2v(checked=checked(), stats=stats_build() and not checked())
        L = ctypes.CDLL(path)
        vp, i64, i32, u64, dbl, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_size_t)
        P = ctypes.POINTER
        L.n2v_tune_default.argtypes = [P(n2v_tune)]
        L.n2v_tune_default.restype = None
        L.n2v_alpha_q16.argtypes = [dbl, dbl, P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.n2v_graph_aux_bytes.argtypes = [i64, i64, ctypes.c_int, P(n2v_tune), P(sz)]
        L.n2v_graph_load.argtypes = [vp, vp, vp, i64, i64, vp, sz, P(n2v_tune), vp, P(vp)]
        L.n2v_graph_info_get.argtypes = [vp, P(n2v_graph_info)]
        L.n2v_graph_retune.argtypes = [vp, P(n2v_tune), vp]
        L.n2v_graph_free.argtypes = [vp]
        L.n2v_graph_free.restype = None
        L.n2v_walk_ws_bytes.argtypes = [vp, i64, i32, ctypes.c_int, P(sz)]
        L.n2v_walk.argtypes = [vp, vp, i64, i32, i32, dbl, dbl, u64, i64, i64, vp, vp, sz, ctypes.c_int, vp]
        L.n2v_walk_traffic.argtypes = [vp, vp, i64, i64, i64, i32, vp, vp, vp]
        L.n2v_walk_noalloc.argtypes = [vp, vp, i64, i32, i32, dbl, dbl, u64, i64, i64, vp, vp]
        L.n2v_walk_stream.argtypes = [vp, vp, i64, i32, i32, dbl, dbl, u64, i64, i64, vp, vp, i64, i32, vp, sz,
                                      ctypes.c_int, vp, vp]
        L.n2v_selftest_timeout.argtypes = [vp, i64, vp]
        L.n2v_walk_approx.argtypes = [vp, vp, i64, i32, i32, dbl, dbl, u64, i64, i64, vp, vp, sz, ctypes.c_int, dbl,
                                      i64, vp]
        L.n2v_stream_status.argtypes = [vp, vp]
        L.n2v_strerror.argtypes = [ctypes.c_int]
        L.n2v_strerror.restype = ctypes.c_char_p
        L.n2v_launch_shape.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.n2v_step_stats.argtypes = [vp, i32, i32]
        L.n2v_serve_cfg_default.argtypes = [P(n2v_serve_cfg)]
        L.n2v_serve_cfg_default.restype = None
        L.n2v_serve_create.argtypes = [vp, vp, sz, P(n2v_serve_cfg), vp, P(vp)]
        L.n2v_serve_submit.argtypes = [vp, P(n2v_job), P(i64)]
        L.n2v_serve_step.argtypes = [vp, P(ctypes.c_int)]
        L.n2v_serve_poll.argtypes = [vp, vp, ctypes.c_int, P(ctypes.c_int)]
        L.n2v_serve_job_rows.argtypes = [vp, i64, P(vp)]
        L.n2v_serve_release.argtypes = [vp, i64]
        L.n2v_serve_stats.argtypes = [vp, P(n2v_serve_stats_t)]
        L.n2v_serve_destroy.argtypes = [vp]
        L.n2v_serve_destroy.restype = None
        L.n2v_stored_bytes.argtypes = [vp, vp, P(sz), P(i64)]
        L.n2v_stored_build.argtypes = [vp, dbl, dbl, vp, sz, vp]
        L.n2v_stored_walk.argtypes = [vp, vp, vp, i64, i32, i32, u64, i64, i64, vp, vp]
        L.n2v_autotune_ws_bytes.argtypes = [vp, i64, i32, P(sz)]
        L.n2v_autotune.argtypes = [vp, vp, i64, i32, dbl, dbl, u64, i64, vp, vp, sz, vp, P(n2v_tune),
                                   P(ctypes.c_float)]
        _LIB = L
    return _LIB


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int, what: str) -> None:
    if rc != N2V_OK:
        raise N2VError(rc, what)


# --------------------------------------------------------------------------
# 1:1 entry points

def n2v_strerror(code: int) -> str:
    return lib().n2v_strerror(code).decode()


def n2v_tune_default() -> n2v_tune:
    t = n2v_tune()
    lib().n2v_tune_default(ctypes.byref(t))
    return t


def n2v_alpha_q16(p: float, q: float) -> tuple[int, int]:
    ap, aq = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().n2v_alpha_q16(p, q, ctypes.byref(ap), ctypes.byref(aq)), "n2v_alpha_q16")
    return ap.value, aq.value


def n2v_graph_aux_bytes(n: int, nnz: int, weighted: bool, tune: n2v_tune | None = None) -> int:
    b = ctypes.c_size_t()
    _check(lib().n2v_graph_aux_bytes(n, nnz, int(weighted), ctypes.byref(tune) if tune else None,
                                     ctypes.byref(b)), "n2v_graph_aux_bytes")
    return b.value


def n2v_graph_load(row_ptr, col, w, n: int, nnz: int, aux, tune: n2v_tune | None = None, stream=None) -> int:
    h = ctypes.c_void_p()
    aux_bytes = aux.numel() * aux.element_size()
    rc = lib().n2v_graph_load(_ptr(row_ptr), _ptr(col), _ptr(w), n, nnz, _ptr(aux), aux_bytes,
                              ctypes.byref(tune) if tune else None, _stream(stream), ctypes.byref(h))
    _check(rc, "n2v_graph_load")
    return h.value


def n2v_graph_info_get(handle: int) -> n2v_graph_info:
    info = n2v_graph_info()
    _check(lib().n2v_graph_info_get(handle, ctypes.byref(info)), "n2v_graph_info_get")
    return info


def n2v_graph_retune(handle: int, tune: n2v_tune, stream=None) -> None:
    _check(lib().n2v_graph_retune(handle, ctypes.byref(tune), _stream(stream)), "n2v_graph_retune")


def n2v_graph_free(handle: int) -> None:
    lib().n2v_graph_free(handle)


def n2v_walk_ws_bytes(handle: int, walk_count: int, l: int, variant: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().n2v_walk_ws_bytes(handle, walk_count, l, variant, ctypes.byref(b)), "n2v_walk_ws_bytes")
    return b.value


def n2v_walk(handle: int, starts, n_starts: int, r: int, l: int, p: float, q: float, seed: int,
             walk_begin: int, walk_count: int, walks, ws, variant: int, stream=None) -> None:
    ws_bytes = 0 if ws is None else ws.numel() * ws.element_size()
    rc = lib().n2v_walk(handle, _ptr(starts), n_starts, r, l, p, q, seed, walk_begin, walk_count, _ptr(walks),
                        _ptr(ws), ws_bytes, variant, _stream(stream))
    _check(rc, "n2v_walk")


def n2v_walk_approx(handle: int, starts, n_starts: int, r: int, l: int, p: float, q: float, seed: int,
                    walk_begin: int, walk_count: int, walks, ws, variant: int, eps: float, popular: int,
                    stream=None) -> None:
    ws_bytes = 0 if ws is None else ws.numel() * ws.element_size()
    rc = lib().n2v_walk_approx(handle, _ptr(starts), n_starts, r, l, p, q, seed, walk_begin, walk_count, _ptr(walks),
                               _ptr(ws), ws_bytes, variant, eps, popular, _stream(stream))
    _check(rc, "n2v_walk_approx")


def n2v_walk_noalloc(handle: int, starts, n_starts: int, r: int, l: int, p: float, q: float, seed: int,
                     walk_begin: int, walk_count: int, walks, stream=None) -> None:
    """The persistent sampler on the library's own scratch: no workspace, no allocation."""
    rc = lib().n2v_walk_noalloc(handle, _ptr(starts), n_starts, r, l, p, q, seed, walk_begin, walk_count,
                                _ptr(walks), _stream(stream))
    _check(rc, "n2v_walk_noalloc")


def n2v_walk_stream(handle: int, starts, n_starts: int, r: int, l: int, p: float, q: float, seed: int,
                    walk_begin: int, walk_count: int, host_walks, dev_ring, ring_walks: int, ring_slots: int, ws,
                    variant: int, stream=None, copy_stream=None) -> None:
    """Walks in chunks through a device ring, each chunk copied to host memory while the next runs."""
    ws_bytes = 0 if ws is None else ws.numel() * ws.element_size()
    cs = None if copy_stream is None else _stream(copy_stream)
    rc = lib().n2v_walk_stream(handle, _ptr(starts), n_starts, r, l, p, q, seed, walk_begin, walk_count,
                               _ptr(host_walks), _ptr(dev_ring), ring_walks, ring_slots, _ptr(ws), ws_bytes, variant,
                               _stream(stream), cs)
    _check(rc, "n2v_walk_stream")


def n2v_walk_traffic(handle: int, starts, n_starts: int, walk_begin: int, walk_count: int, l: int, walks,
                     out2, stream=None) -> None:
    _check(lib().n2v_walk_traffic(handle, _ptr(starts), n_starts, walk_begin, walk_count, l, _ptr(walks),
                                  _ptr(out2), _stream(stream)), "n2v_walk_traffic")


def n2v_selftest_timeout(handle: int, limit_cycles: int, stream=None) -> None:
    _check(lib().n2v_selftest_timeout(handle, limit_cycles, _stream(stream)), "n2v_selftest_timeout")


def n2v_stream_status(handle: int, stream=None) -> int:
    return int(lib().n2v_stream_status(handle, _stream(stream)))


def n2v_launch_shape(handle: int) -> tuple[int, int, int]:
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().n2v_launch_shape(handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "n2v_launch_shape")
    return a.value, b.value, c.value


STAT_NAMES = (["lane_batches", "lane_cycles", "first_batches", "first_cycles"] +
              [f"mode{m}_{f}" for m in range(5) for f in ("steps", "cycles", "short_sum", "long_sum")] +
              ["segments", "spilled_steps", "kernel_warp_cycles", "staged_chunks", "staged_windows",
               "staged_searches", "unused30", "unused31"])


def n2v_step_stats(reset: bool = True) -> dict | None:
    """Step statistics of the stats build as a dict (None in other builds)."""
    out = np.zeros(32, dtype=np.uint64)
    rc = lib().n2v_step_stats(out.ctypes.data, 32, int(reset))
    if rc != N2V_OK:
        return None
    return {name: int(out[i]) for i, name in enumerate(STAT_NAMES)}


def n2v_autotune_ws_bytes(handle: int, sample: int, l: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().n2v_autotune_ws_bytes(handle, sample, l, ctypes.byref(b)), "n2v_autotune_ws_bytes")
    return b.value


def n2v_autotune(handle: int, starts, n_starts: int, l: int, p: float, q: float, seed: int, sample: int, walks,
                 ws, stream=None) -> tuple[n2v_tune, float]:
    best, ms = n2v_tune(), ctypes.c_float()
    ws_bytes = ws.numel() * ws.element_size()
    _check(lib().n2v_autotune(handle, _ptr(starts), n_starts, l, p, q, seed, sample, _ptr(walks), _ptr(ws), ws_bytes,
                              _stream(stream), ctypes.byref(best), ctypes.byref(ms)), "n2v_autotune")
    return best, ms.value


def n2v_stored_bytes(handle: int, stream=None) -> tuple[int, int]:
    """(table buffer bytes, entries) of a stored transition table for this graph (synchronises)."""
    b, e = ctypes.c_size_t(), ctypes.c_int64()
    _check(lib().n2v_stored_bytes(handle, _stream(stream), ctypes.byref(b), ctypes.byref(e)), "n2v_stored_bytes")
    return int(b.value), int(e.value)


def n2v_stored_build(handle: int, p: float, q: float, table, stream=None) -> None:
    nbytes = table.numel() * table.element_size()
    _check(lib().n2v_stored_build(handle, p, q, _ptr(table), nbytes, _stream(stream)), "n2v_stored_build")


def n2v_stored_walk(handle: int, table, starts, n_starts: int, r: int, l: int, seed: int, walk_begin: int,
                    walk_count: int, walks, stream=None) -> None:
    rc = lib().n2v_stored_walk(handle, _ptr(table), _ptr(starts), n_starts, r, l, seed, walk_begin, walk_count,
                               _ptr(walks), _stream(stream))
    _check(rc, "n2v_stored_walk")


def n2v_serve_cfg_default() -> n2v_serve_cfg:
    c = n2v_serve_cfg()
    lib().n2v_serve_cfg_default(ctypes.byref(c))
    return c


def n2v_serve_create(handle: int, arena, cfg: n2v_serve_cfg | None = None, stream=None) -> int:
    out = ctypes.c_void_p()
    nbytes = arena.numel() * arena.element_size()
    _check(lib().n2v_serve_create(handle, _ptr(arena), nbytes, ctypes.byref(cfg) if cfg else None, _stream(stream),
                                  ctypes.byref(out)), "n2v_serve_create")
    return out.value


def n2v_serve_submit(server: int, starts: np.ndarray, l: int, p: float, q: float, seed: int) -> int:
    starts = np.ascontiguousarray(starts, dtype=np.int32)
    job = n2v_job(starts.ctypes.data, starts.shape[0], l, 0, p, q, seed)
    jid = ctypes.c_int64()
    _check(lib().n2v_serve_submit(server, ctypes.byref(job), ctypes.byref(jid)), "n2v_serve_submit")
    return jid.value


def n2v_serve_step(server: int) -> bool:
    launched = ctypes.c_int()
    _check(lib().n2v_serve_step(server, ctypes.byref(launched)), "n2v_serve_step")
    return bool(launched.value)


def n2v_serve_poll(server: int, max_ids: int = 4096) -> list[int]:
    ids = np.zeros(max_ids, dtype=np.int64)
    n = ctypes.c_int()
    _check(lib().n2v_serve_poll(server, ids.ctypes.data, max_ids, ctypes.byref(n)), "n2v_serve_poll")
    return ids[: n.value].tolist()


def n2v_serve_job_rows(server: int, job_id: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().n2v_serve_job_rows(server, job_id, ctypes.byref(p)), "n2v_serve_job_rows")
    return p.value


def n2v_serve_release(server: int, job_id: int) -> None:
    _check(lib().n2v_serve_release(server, job_id), "n2v_serve_release")


def n2v_serve_stats(server: int) -> dict:
    st = n2v_serve_stats_t()
    _check(lib().n2v_serve_stats(server, ctypes.byref(st)), "n2v_serve_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def n2v_serve_destroy(server: int) -> None:
    lib().n2v_serve_destroy(server)


# --------------------------------------------------------------------------
# conveniences

def default_tune(**kw) -> n2v_tune:
    t = n2v_tune_default()
    for k, v in kw.items():
        setattr(t, k, int(v))
    return t


class Graph:
    """A device-resident CSR graph: owns the torch tensors and the aux buffer."""

    def __init__(self, row_ptr, col, w=None, tune: n2v_tune | None = None, device="cuda", stream=None):
        self.row_ptr = torch.as_tensor(row_ptr, dtype=torch.int64).to(device).contiguous()
        self.col = torch.as_tensor(col, dtype=torch.int32).to(device).contiguous()
        if w is not None:
            if isinstance(w, np.ndarray):
                w = torch.from_numpy(np.ascontiguousarray(w).view(np.int32))
            elif w.dtype != torch.int32:
                w = w.view(torch.int32)  # uint32 bits, unchanged
            w = w.to(device).contiguous()
        self.w = w
        self.n = int(self.row_ptr.numel() - 1)
        self.nnz = int(self.col.numel())
        self.tune = tune if tune is not None else n2v_tune_default()
        self.tune_loaded = n2v_tune()  # the tuning the aux buffer is laid out for
        ctypes.pointer(self.tune_loaded)[0] = self.tune
        nbytes = n2v_graph_aux_bytes(self.n, self.nnz, self.w is not None, self.tune)
        self.aux = torch.empty(max(nbytes, 256) // 8 + 32, dtype=torch.int64, device=device)
        self.handle = n2v_graph_load(self.row_ptr, self.col, self.w, self.n, self.nnz, self.aux, self.tune,
                                     stream)

    @classmethod
    def from_csr(cls, csr, tune: n2v_tune | None = None, device="cuda", stream=None) -> "Graph":
        return cls(torch.from_numpy(csr.row_ptr), torch.from_numpy(csr.col), csr.w, tune, device, stream)

    def info(self) -> n2v_graph_info:
        return n2v_graph_info_get(self.handle)

    def retune(self, tune: n2v_tune, stream=None) -> None:
        n2v_graph_retune(self.handle, tune, stream)
        self.tune = tune

    def close(self) -> None:
        if getattr(self, "handle", None):
            n2v_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def walk(graph: Graph, starts, r: int, l: int, p: float, q: float, seed: int, variant: str | int = "persistent",
         walk_begin: int = 0, walk_count: int | None = None, out=None, ws=None, stream=None,
         cuda_graph: bool = False, approx: tuple[float, int] | None = None) -> torch.Tensor:
    """Allocate (if needed) and fill int32 walks [walk_count, l] on the graph's device."""
    dev = graph.row_ptr.device
    starts = torch.as_tensor(starts, dtype=torch.int32).to(dev).contiguous()
    n_starts = int(starts.numel())
    if walk_count is None:
        walk_count = n_starts * r - walk_begin
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    if cuda_graph:
        v |= N2V_FLAG_CUDA_GRAPH
    if out is None:
        out = torch.empty((walk_count, l), dtype=torch.int32, device=dev)
    need = n2v_walk_ws_bytes(graph.handle, walk_count, l, v)
    if need and (ws is None or ws.numel() * ws.element_size() < need):
        ws = torch.empty(need // 8 + 32, dtype=torch.int64, device=dev)
    if approx is not None:
        n2v_walk_approx(graph.handle, starts, n_starts, r, l, p, q, seed, walk_begin, walk_count, out, ws, v,
                        float(approx[0]), int(approx[1]), stream)
    else:
        n2v_walk(graph.handle, starts, n_starts, r, l, p, q, seed, walk_begin, walk_count, out, ws, v, stream)
    return out


def walk_to_host(graph: Graph, starts, r: int, l: int, p: float, q: float, seed: int, ring_walks: int,
                 ring_slots: int = 2, variant: str | int = "persistent", walk_begin: int = 0,
                 walk_count: int | None = None, out=None, stream=None, copy_stream=None) -> torch.Tensor:
    """Walks [walk_count, l] into pinned host memory through a device ring of ring_slots chunks."""
    dev = graph.row_ptr.device
    starts = torch.as_tensor(starts, dtype=torch.int32).to(dev).contiguous()
    n_starts = int(starts.numel())
    if walk_count is None:
        walk_count = n_starts * r - walk_begin
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    if out is None:
        out = torch.empty((walk_count, l), dtype=torch.int32).pin_memory()
    ring = torch.empty((ring_slots, ring_walks, l), dtype=torch.int32, device=dev)
    need = n2v_walk_ws_bytes(graph.handle, ring_walks, l, v)
    ws = torch.empty(need // 8 + 32, dtype=torch.int64, device=dev) if need else None
    if copy_stream is None:
        copy_stream = torch.cuda.Stream(dev)
    n2v_walk_stream(graph.handle, starts, n_starts, r, l, p, q, seed, walk_begin, walk_count, out, ring, ring_walks,
                    ring_slots, ws, v, stream, copy_stream)
    # the ring and workspace are freed on return: let the call's work finish first
    torch.cuda.synchronize(dev)
    return out


def autotune(graph: Graph, starts, l: int, p: float, q: float, seed: int = 1, sample: int = 1 << 16,
             rng_seed: int = 0, stream=None) -> tuple[n2v_tune, float]:
    """Tune the persistent sampler on a random sample of the given start vertices (applied to graph)."""
    dev = graph.row_ptr.device
    starts = torch.as_tensor(starts, dtype=torch.int32).to(dev)
    gen = torch.Generator(device="cpu").manual_seed(rng_seed)
    pick = torch.randperm(starts.numel(), generator=gen)[: min(sample, starts.numel())].to(dev)
    sub = starts[pick].contiguous()
    walks = torch.empty((sub.numel(), l), dtype=torch.int32, device=dev)
    need = n2v_autotune_ws_bytes(graph.handle, sub.numel(), l)
    ws = torch.empty(need // 8 + 32, dtype=torch.int64, device=dev)
    best, ms = n2v_autotune(graph.handle, sub, sub.numel(), l, p, q, seed, sub.numel(), walks, ws, stream)
    graph.tune = best
    return best, ms


class StoredTable:
    """A stored transition table of the graph for one (p, q), in a torch buffer on the graph's device."""

    def __init__(self, graph: Graph, p: float, q: float, stream=None):
        self.graph = graph
        self.p, self.q = p, q
        self.nbytes, self.entries = n2v_stored_bytes(graph.handle, stream)
        self.buf = torch.empty(self.nbytes // 8 + 32, dtype=torch.int64, device=graph.row_ptr.device)
        n2v_stored_build(graph.handle, p, q, self.buf, stream)


def stored_walk(graph: Graph, table: StoredTable, starts, r: int, l: int, seed: int, walk_begin: int = 0,
                walk_count: int | None = None, out=None, stream=None) -> torch.Tensor:
    """Walks [walk_count, l] sampled from a stored table (same rows as walk() with the table's p, q)."""
    dev = graph.row_ptr.device
    starts = torch.as_tensor(starts, dtype=torch.int32).to(dev).contiguous()
    n_starts = int(starts.numel())
    if walk_count is None:
        walk_count = n_starts * r - walk_begin
    if out is None:
        out = torch.empty((walk_count, l), dtype=torch.int32, device=dev)
    n2v_stored_walk(graph.handle, table.buf, starts, n_starts, r, l, seed, walk_begin, walk_count, out, stream)
    return out


def traffic(graph: Graph, starts, walk_begin: int, walks: torch.Tensor, stream=None) -> tuple[int, int, int]:
    """(real transitions, model adjacency bytes, lower-model bytes) of the rows in ``walks`` (synchronises)."""
    dev = graph.row_ptr.device
    starts = torch.as_tensor(starts, dtype=torch.int32).to(dev).contiguous()
    out3 = torch.zeros(3, dtype=torch.int64, device=dev)
    n2v_walk_traffic(graph.handle, starts, int(starts.numel()), walk_begin, int(walks.shape[0]),
                     int(walks.shape[1]), walks, out3, stream)
    o = out3.cpu()
    return int(o[0]), int(o[1]), int(o[2])


class Server:
    """Continuous-batching walk server over a Graph; the arena is a torch buffer."""

    def __init__(self, graph: Graph, arena_bytes: int, cfg: n2v_serve_cfg | None = None, stream=None):
        self.graph = graph
        self.arena = torch.empty(arena_bytes // 8 + 64, dtype=torch.int64, device=graph.row_ptr.device)
        self.stream = stream
        self.handle = n2v_serve_create(graph.handle, self.arena, cfg, stream)
        self.jobs: dict[int, tuple[int, int]] = {}

    def submit(self, starts, l: int, p: float, q: float, seed: int) -> int:
        starts = np.ascontiguousarray(starts, dtype=np.int32)
        jid = n2v_serve_submit(self.handle, starts, l, p, q, seed)
        self.jobs[jid] = (starts.shape[0], l)
        return jid

    def step(self) -> bool:
        return n2v_serve_step(self.handle)

    def poll(self) -> list[int]:
        return n2v_serve_poll(self.handle)

    def rows(self, jid: int) -> torch.Tensor:
        """A view of a finished job's rows inside the arena (valid until release)."""
        ptr = n2v_serve_job_rows(self.handle, jid)
        n, l = self.jobs[jid]
        off = (ptr - self.arena.data_ptr()) // 4
        return self.arena.view(torch.int32)[off: off + n * l].view(n, l)

    def release(self, jid: int) -> None:
        n2v_serve_release(self.handle, jid)
        self.jobs.pop(jid, None)

    def stats(self) -> dict:
        return n2v_serve_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            n2v_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
