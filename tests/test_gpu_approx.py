"""FN-Approx on the GPU equals the oracle's FN-Approx row for row (needs a GB300).

The approximation changes the walks (it is not the exact node2vec
distribution), but its decision is made in the same IEEE-double formula on
both sides, so the approximate rows are still bit-exact between the CUDA
samplers and the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu

VARIANTS = ["plain", "binned", "persistent"]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("eps,popular", [(1e-2, 256), (1e-3, 64), (0.0, 64)])
def test_approx_rows_match_oracle(weighted, eps, popular):
    g = G.rmat(14, 16, 0.57, 0.19, 0.19, 6)
    if weighted:
        g = G.with_weights(g, 2, 1, 100)
    starts = np.arange(g.n, dtype=np.int32)
    ids = np.arange(g.n * 2)
    want, n_approx, _ = oracle.walk_approx(g.row_ptr, g.col, g.w, starts, 30, 0.5, 2.0, 12, ids, eps, popular,
                                           threads=8)
    if eps > 0 and not weighted:
        assert n_approx > 0
    for tname in [{}, dict(thread_max_deg=0, stream_ratio=0), dict(thread_max_deg=0, stage_window=64,
                                                                    stream_ratio=100_000)]:
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**tname))
        for v in VARIANTS:
            got = n2v.walk(graph, starts, 2, 30, 0.5, 2.0, 12, v, approx=(eps, popular)).cpu().numpy()
            assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
            np.testing.assert_array_equal(got, want, err_msg=f"{tname} {v}")
    if eps == 0.0:
        exact = oracle.walk(g.row_ptr, g.col, g.w, starts, 30, 0.5, 2.0, 12, ids, threads=8)
        np.testing.assert_array_equal(want, exact)


def test_approx_rejects_bad_arguments():
    g = G.rmat(10, 8, 0.57, 0.19, 0.19, 1)
    graph = n2v.Graph.from_csr(g)
    with pytest.raises(n2v.N2VError):
        n2v.walk(graph, [0], 1, 4, 1.0, 1.0, 1, "persistent", approx=(-1.0, 10))
    with pytest.raises(n2v.N2VError):
        n2v.walk(graph, [0], 1, 4, 1.0, 1.0, 1, "persistent", approx=(1e-3, 0))
