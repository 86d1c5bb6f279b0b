"""Autotuner results kept on disk, per graph, GPU, library build and tuning sample.

``n2v_autotune`` times candidate tunings of the persistent sampler on a sample of the job. On
R-MAT 26 that takes about 13 s. A second run of the same job on the same kind of GPU would find
the same tuning, so this module keeps the result in a directory, one small JSON file per key,
and applies it on the next run instead of tuning again.

What the key covers:
- the graph: vertex and edge counts, whether it is weighted, all of ``row_ptr``, and a fixed
  sample of ``col`` (and of the weights): up to 4,096 blocks of 4 KB at an even stride;
- the GPU: its name, SM count, compute capability and memory size;
- the library build: the digest ``_build`` stamps ``libn2v.so`` with (sources, flags, machine);
- the sample the tuner timed: walk length, p, q, seed, sample size, and the tuning it started
  from.

A tuning never changes a row: the tunables choose how the work is scheduled, not what is
computed. So a stale or colliding entry can cost speed but cannot change a walk. That is why the
key may sample ``col`` instead of hashing all 8.4 GB of it on R-MAT 26.
"""
from __future__ import annotations

import hashlib
import json
import os
import struct
import tempfile

import numpy as np

BLOCK_BYTES = 4096
MAX_BLOCKS = 4096


def _sample_blocks(h, a: np.ndarray) -> None:
    """Feed up to MAX_BLOCKS blocks of BLOCK_BYTES of the array's bytes, at an even stride, to h."""
    b = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    n = b.size
    h.update(struct.pack("<q", n))
    nblocks = (n + BLOCK_BYTES - 1) // BLOCK_BYTES
    if nblocks <= MAX_BLOCKS:
        h.update(b.tobytes())
        return
    stride = nblocks // MAX_BLOCKS
    for i in range(MAX_BLOCKS):
        off = i * stride * BLOCK_BYTES
        h.update(b[off:off + BLOCK_BYTES].tobytes())
    h.update(b[max(0, n - BLOCK_BYTES):].tobytes())  # and the tail


def graph_fingerprint(row_ptr, col, w=None) -> str:
    """Fingerprint of a CSR graph: counts, all of row_ptr, and a fixed sample of col and w."""
    row_ptr = np.asarray(row_ptr)
    col = np.asarray(col)
    h = hashlib.sha256()
    h.update(struct.pack("<qqB", row_ptr.size - 1, col.size, 0 if w is None else 1))
    h.update(np.ascontiguousarray(row_ptr, dtype=np.int64).tobytes())
    _sample_blocks(h, np.ascontiguousarray(col, dtype=np.int32))
    if w is not None:
        _sample_blocks(h, np.ascontiguousarray(np.asarray(w)).view(np.uint32))
    return h.hexdigest()[:32]


def device_key(device=None) -> dict:
    """The GPU's identity as far as the tuning is concerned."""
    import torch

    p = torch.cuda.get_device_properties(device if device is not None else torch.cuda.current_device())
    return {"name": p.name, "sms": p.multi_processor_count, "cc": [p.major, p.minor],
            "mem_gb": round(p.total_memory / 2**30)}


def library_key() -> str:
    """The digest libn2v.so was built from (its in-tree stamp)."""
    from . import _build

    try:
        with open(_build.LIBN2V + ".stamp") as f:
            return f.read().strip()[:32]
    except OSError:
        return "unbuilt"


def entry_key(graph_fp: str, device: dict, library: str, l: int, p: float, q: float, seed: int, sample: int,
              base_tune: dict) -> str:
    spec = {"graph": graph_fp, "device": device, "library": library, "l": int(l), "p": float(p), "q": float(q),
            "seed": int(seed), "sample": int(sample), "base_tune": {k: int(v) for k, v in sorted(base_tune.items())}}
    return hashlib.sha256(json.dumps(spec, sort_keys=True).encode()).hexdigest()[:40]


class TuneCache:
    """A directory of tuned results, one JSON file per key."""

    def __init__(self, directory: str):
        self.dir = directory
        os.makedirs(directory, exist_ok=True)

    def _path(self, key: str) -> str:
        return os.path.join(self.dir, f"tune_{key}.json")

    def get(self, key: str) -> dict | None:
        """The stored entry ({"tune": {...}, "sample_ms": ..., ...}), or None (also for an unreadable file)."""
        try:
            with open(self._path(key)) as f:
                d = json.load(f)
        except (OSError, ValueError):
            return None
        if not isinstance(d, dict) or not isinstance(d.get("tune"), dict):
            return None
        return d

    def put(self, key: str, tune: dict, sample_ms: float, meta: dict | None = None) -> str:
        """Store an entry atomically (written to a temporary file, then renamed)."""
        d = {"tune": {k: int(v) for k, v in tune.items()}, "sample_ms": float(sample_ms), **(meta or {})}
        fd, tmp = tempfile.mkstemp(dir=self.dir, prefix=".tune_", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(tmp, self._path(key))
        return self._path(key)


def autotune_cached(cache: TuneCache, graph, csr, starts, l: int, p: float, q: float, seed: int = 1,
                    sample: int = 1 << 16, stream=None, n2v_mod=None) -> tuple[object, float, bool]:
    """n2v.autotune, or its stored result for the same key applied with graph.retune.

    Returns (tuning, sample time in ms as measured when it was tuned, whether it came from the cache).
    """
    if n2v_mod is None:
        from . import n2v as n2v_mod
    base = graph.tune.as_dict()
    key = entry_key(graph_fingerprint(csr.row_ptr, csr.col, csr.w), device_key(graph.row_ptr.device),
                    library_key(), l, p, q, seed, sample, base)
    hit = cache.get(key)
    if hit is not None:
        tune = n2v_mod.default_tune(**hit["tune"])
        graph.retune(tune, stream)
        return tune, float(hit["sample_ms"]), True
    tune, ms = n2v_mod.autotune(graph, starts, l, p, q, seed, sample=sample, stream=stream)
    cache.put(key, tune.as_dict(), ms, {"l": int(l), "p": float(p), "q": float(q), "sample": int(sample)})
    return tune, ms, False
