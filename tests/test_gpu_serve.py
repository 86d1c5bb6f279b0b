"""Autotuner and serving loop on the GPU (needs a GB300).

* The autotuner returns a valid tuning and the rows under it are still the
  oracle's.
* The serving loop admits jobs by free arena memory, mixes them into ticks,
  and every job's rows equal the same job run alone through n2v_walk (and,
  for a sample, the oracle) -- the same alone and in the mix.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.fixture(scope="module")
def rmat15():
    return G.rmat(15, 16, 0.57, 0.19, 0.19, 5)


def test_autotune_keeps_rows_exact(rmat15):
    g = rmat15
    graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(hub_count=64))
    starts = np.arange(g.n, dtype=np.int32)
    best, ms = n2v.autotune(graph, starts, 20, 0.5, 2.0, sample=8192)
    assert ms > 0 and best.stage_window in (0, 256, 512, 1024) and best.blocks_per_sm in (4, 5, 6)
    if best.hub_count == 0:
        assert graph.info().hub_count == 0
    ids = np.arange(0, g.n * 2, 5)
    got = n2v.walk(graph, starts, 2, 20, 0.5, 2.0, 3, "persistent").cpu().numpy()[ids]
    want = oracle.walk(g.row_ptr, g.col, None, starts, 20, 0.5, 2.0, 3, ids, threads=8)
    np.testing.assert_array_equal(got, want)


def q16(x):
    return round(x * 65536) / 65536


def make_jobs(n_vertices, count, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        size = int(np.exp(rng.uniform(0, np.log(3000))))
        starts = rng.integers(0, n_vertices, size=size).astype(np.int32)
        l = int(rng.choice([10, 20, 40, 80]))
        p = q16(float(np.exp(rng.uniform(np.log(0.25), np.log(4)))))
        q = q16(float(np.exp(rng.uniform(np.log(0.25), np.log(4)))))
        jobs.append((starts, l, p, q, 1000 + j))
    return jobs


def test_serving_mix_equals_alone(rmat15):
    g = rmat15
    graph = n2v.Graph.from_csr(g)
    jobs = make_jobs(g.n, 48, 7)
    cfg = n2v.n2v_serve_cfg_default()
    cfg.tick_walkers = 8192
    cfg.min_share = 512
    cfg.spill_specials = 32
    # a small arena (about 2.4 MB for jobs after the tick tables): admission has
    # to wait for memory to free up
    srv = n2v.Server(graph, 3 << 20, cfg)
    ids, order = {}, []
    saw_queue = False
    for i, (starts, l, p, q, seed) in enumerate(jobs):
        ids[srv.submit(starts, l, p, q, seed)] = i
        if i % 12 == 11:  # jobs keep arriving while earlier ones run
            srv.step()
            saw_queue |= srv.stats()["queued"] > 0
    done = 0
    checked_oracle = 0
    for _ in range(100_000):
        srv.step()
        st = srv.stats()
        saw_queue |= st["queued"] > 0
        for jid in srv.poll():
            starts, l, p, q, seed = jobs[ids[jid]]
            got = srv.rows(jid).clone()
            alone = n2v.walk(graph, starts, 1, l, p, q, seed, "persistent")
            assert torch.equal(got, alone), f"job {ids[jid]} differs from the same job alone"
            if checked_oracle < 6 and starts.size <= 400:
                want = oracle.walk(g.row_ptr, g.col, None, starts, l, p, q, seed, np.arange(starts.size), threads=8)
                np.testing.assert_array_equal(got.cpu().numpy(), want)
                checked_oracle += 1
            order.append(ids[jid])
            srv.release(jid)
            done += 1
        if done == len(jobs):
            break
    assert done == len(jobs)
    assert saw_queue, "the arena never limited admission"
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    assert srv.stats()["arena_used"] == 0
    srv.close()


def test_serving_rejects_oversized_and_bad_jobs(rmat15):
    graph = n2v.Graph.from_csr(rmat15)
    cfg = n2v.n2v_serve_cfg_default()
    cfg.spill_specials = 0
    srv = n2v.Server(graph, 1 << 20, cfg)
    with pytest.raises(n2v.N2VError):
        srv.submit(np.zeros(100_000, dtype=np.int32), 80, 1.0, 1.0, 1)  # can never fit
    with pytest.raises(n2v.N2VError):
        srv.submit(np.zeros(10, dtype=np.int32), 10, 0.0, 1.0, 1)  # p must be > 0
    srv.close()
