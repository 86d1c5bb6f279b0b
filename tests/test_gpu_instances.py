"""The persistent sampler's instances give the same rows (needs a GB300).

The host compiles the persistent kernel as a full instance and as two lean ones. The lean ones
leave out the hub caches, the merge form and FN-Approx; one of them also leaves out the weighted
paths. For an exact walk without hub caches or the merge form it picks a lean instance. FN-Approx
with eps = 0 walks exactly but always takes the full instance. So the two calls below run the
same rows through different instances, at every compiled register budget, and both must equal
the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu

TUNES = [
    {},
    dict(thread_max_deg=0),
    dict(thread_max_deg=0, stage_window=64, stream_ratio=100_000),
    dict(blocks_per_sm=4),
    dict(blocks_per_sm=6),
    dict(blocks_per_sm=8),
]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.mark.parametrize("weighted", [False, True])
def test_lean_and_full_instances_agree(weighted):
    g = G.rmat(14, 16, 0.57, 0.19, 0.19, 3)
    if weighted:
        g = G.with_weights(g, 2, 1, 100)
    starts = np.arange(g.n, dtype=np.int32)
    want = oracle.walk(g.row_ptr, g.col, g.w, starts, 30, 2.0, 0.5, 5, np.arange(g.n), threads=8)
    for tname in TUNES:
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**tname))
        lean = n2v.walk(graph, starts, 1, 30, 2.0, 0.5, 5, "persistent").cpu().numpy()
        full = n2v.walk(graph, starts, 1, 30, 2.0, 0.5, 5, "persistent", approx=(0.0, 64)).cpu().numpy()
        assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
        np.testing.assert_array_equal(lean, want, err_msg=f"lean {tname}")
        np.testing.assert_array_equal(full, want, err_msg=f"full {tname}")
