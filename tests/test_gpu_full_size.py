"""Full-size configs in the launch configuration bench.py times (needs a GB300).

* R-MAT scale 26 (one walk per vertex, l = 80, p = 2, q = 0.5): the whole job
  through the persistent sampler in launches of 2^23 walks, recorded as a CUDA
  graph on a side stream, as the bench runs it.  Sampled rows (random walk ids
  plus the walks from the 100 largest hubs) match the oracle.
* Serving on R-MAT scale 24: the first jobs of the bench's job mix, served
  together through one server; every job equals the same job run alone, and
  sampled rows of each match the oracle.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()
    yield
    torch.cuda.synchronize()


def test_rmat26_full_job_sampled_rows():
    wl = G.WORKLOADS["rmat26"]
    g = G.workload_graph("rmat26")
    graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**bench.WORKLOAD_DEFAULTS["rmat26"]["tune"]))
    starts = np.arange(g.n, dtype=np.int32)
    p, q = wl.pq[0]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        out = n2v.walk(graph, starts, wl.r, wl.l, p, q, wl.seed, "persistent", cuda_graph=True)
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    assert out.shape == (g.n * wl.r, wl.l)
    rng = np.random.default_rng(26)
    hubs = np.argsort(-g.degrees(), kind="stable")[:100]
    ids = np.unique(np.concatenate([rng.choice(g.n * wl.r, size=8192, replace=False), hubs]))
    want = oracle.walk(g.row_ptr, g.col, None, starts, wl.l, p, q, wl.seed, ids, threads=16)
    got = out[torch.from_numpy(ids).cuda()].cpu().numpy()
    np.testing.assert_array_equal(got, want)
    del out


def test_rmat24_serving_mix_equals_alone():
    g = G.workload_graph("rmat24serve")
    graph = n2v.Graph.from_csr(g)
    jobs = [jb for jb in bench.serving_jobs(g.n, 200) if jb["size"] <= 1 << 16][:40]
    for jb in jobs:
        jb["starts"] = G.uniform(jb["seed"], jb["stream"], g.n, jb["size"]).astype(np.int32)
    srv = n2v.Server(graph, 8 << 30)
    ids = {srv.submit(jb["starts"], jb["l"], jb["p"], jb["q"], jb["seed"]): i for i, jb in enumerate(jobs)}
    done, rng = 0, np.random.default_rng(24)
    for _ in range(1_000_000):
        srv.step()
        for jid in srv.poll():
            jb = jobs[ids[jid]]
            got = srv.rows(jid).clone()
            alone = n2v.walk(graph, jb["starts"], 1, jb["l"], jb["p"], jb["q"], jb["seed"], "persistent")
            assert torch.equal(got, alone), f"job {ids[jid]} differs from the same job alone"
            sel = np.sort(rng.choice(jb["size"], size=min(64, jb["size"]), replace=False))
            want = oracle.walk(g.row_ptr, g.col, None, jb["starts"], jb["l"], jb["p"], jb["q"], jb["seed"], sel,
                               threads=16)
            np.testing.assert_array_equal(got[torch.from_numpy(sel).cuda()].cpu().numpy(), want)
            srv.release(jid)
            done += 1
        if done == len(jobs):
            break
    assert done == len(jobs)
    assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
    srv.close()
