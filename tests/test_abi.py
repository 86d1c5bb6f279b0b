"""The C-ABI library builds, loads and exports every declared entry point (no GPU).

Only host-side logic runs here: argument checks that return before any CUDA
call, the Q16 rounding, status strings and buffer sizing.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1805_00280_gb300 import n2v

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(REPO, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(REPO, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(n2v_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = n2v.lib()
    names = declared_functions()
    assert len(names) >= 12
    missing = [nm for nm in names if not hasattr(L, nm)]
    assert not missing, missing


def test_alpha_q16_matches_oracle():
    rng = np.random.default_rng(11)
    cases = [(1.0, 1.0), (0.5, 2.0), (0.25, 4.0), (4.0, 0.25), (3.0, 0.3), (2.0**-8, 65536.0)]
    cases += [(float(np.exp(a)), float(np.exp(b))) for a, b in rng.uniform(-4, 4, size=(3000, 2))]
    for p, q in cases:
        assert n2v.n2v_alpha_q16(p, q) == oracle.alpha_q16(p, q)


@pytest.mark.parametrize("p,q", [(0.0, 1.0), (1.0, -2.0), (math.nan, 1.0), (1.0, math.inf), (1e6, 1.0),
                                 (1.0, 1e-9)])
def test_alpha_q16_rejects(p, q):
    with pytest.raises(n2v.N2VError) as e:
        n2v.n2v_alpha_q16(p, q)
    assert e.value.code == n2v.N2V_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        oracle.alpha_q16(p, q)


def test_strerror_covers_codes():
    for code in range(-7, 1):
        assert n2v.n2v_strerror(code) != "unknown status"
    assert n2v.n2v_strerror(42) == "unknown status"


def test_aux_bytes_sizing():
    t = n2v.n2v_tune_default()
    assert t.block_threads % 32 == 0 and t.smem_specials >= 32
    a = n2v.n2v_graph_aux_bytes(1000, 10_000, False, t)
    b = n2v.n2v_graph_aux_bytes(1000, 10_000, True, t)
    assert b - a >= 8 * 10_000  # the static weight prefix
    t.hub_count = 16
    c = n2v.n2v_graph_aux_bytes(1000, 10_000, False, t)
    assert c - a >= 4 * 1000  # per-vertex hub index
    t.hub_count = 0
    t.bitmap_hubs = 8
    d = n2v.n2v_graph_aux_bytes(1000, 10_000, False, t)
    assert d - a >= 8 * 16 * ((1000 + 63) // 64)  # 16 bytes per 64 vertices per bitmap hub
    t.reserved[0] = 1
    with pytest.raises(n2v.N2VError):
        n2v.n2v_graph_aux_bytes(1000, 10_000, False, t)
    with pytest.raises(n2v.N2VError):
        n2v.n2v_graph_aux_bytes(0, 10, False, None)


def test_host_argument_checks_need_no_gpu():
    L = n2v.lib()
    out = ctypes.c_void_p()
    assert L.n2v_graph_load(None, None, None, 10, 0, None, 0, None, None, ctypes.byref(out)) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_walk(None, None, 1, 1, 1, 1.0, 1.0, 1, 0, 1, None, None, 0, 0, None) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_stream_status(None, None) == n2v.N2V_ERR_INVALID_ARG
    b = ctypes.c_size_t()
    assert L.n2v_walk_ws_bytes(None, 1, 1, 0, ctypes.byref(b)) == n2v.N2V_ERR_INVALID_ARG
    L.n2v_graph_free(None)  # no-op


@pytest.mark.parametrize("field,value", [("block_threads", 512), ("block_threads", 48), ("block_threads", 32),
                                         ("stage_window", 100), ("stage_window", 8192), ("stage_buffers", 3),
                                         ("smem_specials", 48), ("smem_specials", 16), ("stream_ratio", -1),
                                         ("blocks_per_sm", -1), ("hub_budget_mb", -1), ("bitmap_hubs", -1),
                                         ("bitmap_hubs", 4097), ("block_min_deg", -1), ("merge_ratio", -1),
                                         ("l2_persist_mb", -1), ("l2_persist_mb", 5000)])
def test_tune_validation_rejects(field, value):
    t = n2v.n2v_tune_default()
    setattr(t, field, value)
    with pytest.raises(n2v.N2VError):
        n2v.n2v_graph_aux_bytes(1000, 10_000, False, t)


@pytest.mark.parametrize("field,value", [("block_threads", 64), ("block_threads", 256), ("stage_window", 0),
                                         ("stage_window", 4096), ("stage_buffers", 4), ("blocks_per_sm", 8),
                                         ("bitmap_hubs", 64), ("block_min_deg", 1), ("block_min_deg", 1 << 30),
                                         ("merge_ratio", 0), ("merge_ratio", 1000), ("l2_persist_mb", 64)])
def test_tune_validation_accepts(field, value):
    t = n2v.n2v_tune_default()
    setattr(t, field, value)
    assert n2v.n2v_graph_aux_bytes(1000, 10_000, False, t) > 0


def test_stored_serve_and_tuner_host_checks_need_no_gpu():
    L = n2v.lib()
    b, e = ctypes.c_size_t(), ctypes.c_int64()
    assert L.n2v_stored_bytes(None, None, ctypes.byref(b), ctypes.byref(e)) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_stored_build(None, 1.0, 1.0, None, 0, None) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_stored_walk(None, None, None, 1, 1, 1, 1, 0, 1, None, None) == n2v.N2V_ERR_INVALID_ARG
    srv = ctypes.c_void_p()
    assert L.n2v_serve_create(None, None, 0, None, None, ctypes.byref(srv)) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_autotune_ws_bytes(None, 1, 1, ctypes.byref(b)) == n2v.N2V_ERR_INVALID_ARG
    assert L.n2v_walk_traffic(None, None, 1, 0, 0, 1, None, None, None) == n2v.N2V_ERR_INVALID_ARG


def test_step_stats_report_nothing_outside_the_stats_build():
    """n2v_step_stats is a stats-build tool: the product library fills zeros and says so, without a device."""
    import numpy as np

    L = n2v.lib()
    out = np.full(32, 7, dtype=np.uint64)
    assert L.n2v_step_stats(out.ctypes.data, 33, 0) == n2v.N2V_ERR_INVALID_ARG
    if not n2v.stats_build():
        assert L.n2v_step_stats(out.ctypes.data, 32, 0) == n2v.N2V_ERR_INVALID_ARG
        assert not out.any()
        assert n2v.n2v_step_stats() is None
