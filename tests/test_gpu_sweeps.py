"""GPU parity on the shapes of the paper's synthetic sweeps (Section 4.1): the
Skew-S graphs (R-MAT with b = c = 0.25 and d = S a; here S = 5, the most
skewed) and the WeC-K graphs (R-MAT (0.18, 0.25, 0.25, 0.32)), both with the
sweep's 50 generated edges per vertex, at scale 16 so that the oracle checks
thousands of rows in seconds.  One walk of length 80 per vertex at
p = 0.5, q = 2, as in the sweeps; the persistent sampler in its default
tuning, with rank bitmaps and with the block tier, and the binned sampler,
against the oracle on random walk ids plus every walk that starts at one of
the 64 largest hubs.  Needs a GB300.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_00280_gb300 import graphs as G
from paper_1805_00280_gb300 import n2v

pytestmark = pytest.mark.gpu

SHAPES = {
    "skew5_s16": dict(kind="rmat", scale=16, ef=50, seed=1, abc=G.skew_abc(5)),
    "wec_s16": dict(kind="rmat", scale=16, ef=50, seed=1, abc=(0.18, 0.25, 0.25)),
}
TUNES = {
    "default": {},
    "bitmaps": dict(bitmap_hubs=64),
    "block": dict(block_min_deg=512),
    "block_bitmaps_stage": dict(block_min_deg=256, bitmap_hubs=16, stream_ratio=1000, stage_window=256),
}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    n2v.lib()


@pytest.mark.parametrize("shape", list(SHAPES))
def test_sweep_shape_rows_match_oracle(shape):
    g = G.make_graph(SHAPES[shape])
    starts = np.arange(g.n, dtype=np.int32)
    l, p, q, seed = 80, 0.5, 2.0, 1
    rng = np.random.default_rng(16)
    hubs = np.argsort(-g.degrees(), kind="stable")[:64]
    ids = np.unique(np.concatenate([rng.choice(g.n, size=3000, replace=False), hubs]))
    want = oracle.walk(g.row_ptr, g.col, None, starts, l, p, q, seed, ids, threads=16)
    ref = None
    for tname, tune in TUNES.items():
        graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**tune))
        for variant in (["persistent", "binned"] if tname == "default" else ["persistent"]):
            out = n2v.walk(graph, starts, 1, l, p, q, seed, variant)
            assert n2v.n2v_stream_status(graph.handle) == n2v.N2V_OK
            np.testing.assert_array_equal(out[torch.from_numpy(ids).cuda()].cpu().numpy(), want,
                                          err_msg=f"{shape} {tname} {variant}")
            if ref is None:
                ref = out
            else:  # every tuning gives the same full output
                assert torch.equal(out, ref), f"{shape} {tname} {variant}"
        graph.close()
