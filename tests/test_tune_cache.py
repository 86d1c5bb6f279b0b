"""The on-disk store of autotuner results (host logic, no GPU)."""
import json
import types

import numpy as np

from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import tune_cache as tc


def small_graph():
    return G.rmat(12, 8, 0.57, 0.19, 0.19, 2)


def test_fingerprint_is_stable_and_sees_changes():
    g = small_graph()
    a = tc.graph_fingerprint(g.row_ptr, g.col)
    assert a == tc.graph_fingerprint(g.row_ptr.copy(), g.col.copy())
    col = g.col.copy()
    col[5] ^= 1
    assert tc.graph_fingerprint(g.row_ptr, col) != a  # small arrays are hashed whole
    rp = g.row_ptr.copy()
    rp[1:-1] += 0  # unchanged
    assert tc.graph_fingerprint(rp, g.col) == a
    w = np.ones(g.col.size, dtype=np.uint32)
    assert tc.graph_fingerprint(g.row_ptr, g.col, w) != a
    w2 = w.copy()
    w2[0] = 2
    assert tc.graph_fingerprint(g.row_ptr, g.col, w2) != tc.graph_fingerprint(g.row_ptr, g.col, w)


def test_fingerprint_samples_large_lists():
    """Past MAX_BLOCKS blocks only a strided sample (and the tail) of col is hashed."""
    n_blocks = tc.MAX_BLOCKS * 3
    col = np.arange(n_blocks * tc.BLOCK_BYTES // 4, dtype=np.int32)
    rp = np.array([0, col.size], dtype=np.int64)
    base = tc.graph_fingerprint(rp, col)
    sampled = col.copy()
    sampled[0] += 1  # block 0 is sampled
    assert tc.graph_fingerprint(rp, sampled) != base
    tail = col.copy()
    tail[-1] += 1  # the tail is sampled
    assert tc.graph_fingerprint(rp, tail) != base
    skipped = col.copy()
    skipped[tc.BLOCK_BYTES // 4] += 1  # block 1 lies between two sampled blocks (stride 3)
    assert tc.graph_fingerprint(rp, skipped) == base


def test_entry_key_covers_every_field():
    dev = {"name": "GPU", "sms": 152, "cc": [10, 3], "mem_gb": 277}
    args = dict(graph_fp="abc", device=dev, library="lib", l=20, p=2.0, q=0.5, seed=1, sample=1 << 20,
                base_tune={"stream_ratio": 40, "chunk_walkers": 0})
    k = tc.entry_key(**args)
    assert k == tc.entry_key(**dict(args, base_tune={"chunk_walkers": 0, "stream_ratio": 40}))  # order-free
    for field, other in [("graph_fp", "abd"), ("device", dict(dev, sms=148)), ("library", "lib2"), ("l", 80),
                         ("p", 1.0), ("q", 1.0), ("seed", 2), ("sample", 1 << 16),
                         ("base_tune", {"stream_ratio": 100, "chunk_walkers": 0})]:
        assert tc.entry_key(**dict(args, **{field: other})) != k, field


def test_store_roundtrip_and_bad_files(tmp_path):
    c = tc.TuneCache(str(tmp_path / "cache"))
    assert c.get("k1") is None
    p = c.put("k1", {"stream_ratio": 100, "blocks_per_sm": 5}, 12.5, {"l": 20})
    d = c.get("k1")
    assert d["tune"] == {"stream_ratio": 100, "blocks_per_sm": 5} and d["sample_ms"] == 12.5 and d["l"] == 20
    assert json.load(open(p)) == d
    (tmp_path / "cache" / "tune_k2.json").write_text("{not json")
    assert c.get("k2") is None
    (tmp_path / "cache" / "tune_k3.json").write_text(json.dumps({"tune": 5}))
    assert c.get("k3") is None
    assert not [f for f in (tmp_path / "cache").iterdir() if f.name.startswith(".tune_")]  # no temporaries left


class FakeTune(dict):
    def as_dict(self):
        return dict(self)


def fake_n2v(calls):
    def autotune(graph, starts, l, p, q, seed, sample, stream=None):
        calls.append(("autotune", l, p, q, seed, sample))
        t = FakeTune(graph.tune, stream_ratio=100)
        graph.tune = t
        return t, 7.5

    return types.SimpleNamespace(autotune=autotune, default_tune=lambda **kw: FakeTune(kw))


def fake_graph(base):
    g = types.SimpleNamespace(tune=FakeTune(base), row_ptr=types.SimpleNamespace(device=None), retuned=[])
    g.retune = lambda t, stream=None: (g.retuned.append(dict(t)), setattr(g, "tune", t))
    return g


def test_autotune_cached_miss_then_hit(tmp_path, monkeypatch):
    monkeypatch.setattr(tc, "device_key", lambda device=None: {"name": "GPU", "sms": 152})
    monkeypatch.setattr(tc, "library_key", lambda: "lib")
    csr = small_graph()
    cache = tc.TuneCache(str(tmp_path))
    calls = []
    base = {"stream_ratio": 40, "chunk_walkers": 0}
    g1 = fake_graph(base)
    t, ms, hit = tc.autotune_cached(cache, g1, csr, np.arange(csr.n), 20, 2.0, 0.5, 1, 4096, n2v_mod=fake_n2v(calls))
    assert not hit and ms == 7.5 and t["stream_ratio"] == 100 and len(calls) == 1
    g2 = fake_graph(base)
    t, ms, hit = tc.autotune_cached(cache, g2, csr, np.arange(csr.n), 20, 2.0, 0.5, 1, 4096, n2v_mod=fake_n2v(calls))
    assert hit and ms == 7.5 and len(calls) == 1  # not tuned again
    assert g2.retuned == [{"stream_ratio": 100, "chunk_walkers": 0}] and g2.tune["stream_ratio"] == 100
    # another sample size, another start tuning or another graph: tuned again
    tc.autotune_cached(cache, fake_graph(base), csr, np.arange(csr.n), 20, 2.0, 0.5, 1, 2048, n2v_mod=fake_n2v(calls))
    tc.autotune_cached(cache, fake_graph(dict(base, chunk_walkers=1 << 23)), csr, np.arange(csr.n), 20, 2.0, 0.5, 1,
                       4096, n2v_mod=fake_n2v(calls))
    other = G.rmat(12, 8, 0.57, 0.19, 0.19, 3)
    tc.autotune_cached(cache, fake_graph(base), other, np.arange(other.n), 20, 2.0, 0.5, 1, 4096,
                       n2v_mod=fake_n2v(calls))
    assert len(calls) == 4
