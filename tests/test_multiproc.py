"""Walk-id sharding over ranks, tested with world_size-2 gloo process groups on CPU.

Each rank computes its shard of a job (the CPU oracle stands in for the
per-rank device sampler, whose rows equal the oracle's); the shards gathered
over gloo must equal one process computing the whole job, and the timing
reduction takes the slowest rank.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_00280_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, mode, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1805_00280_gb300 import graphs as G

    g = G.rmat(11, 8, 0.57, 0.19, 0.19, 4)
    starts = np.arange(g.n, dtype=np.int32)
    l, p, q, seed = 12, 0.5, 2.0, 9
    if mode == "weak":
        r_total, begin, count = shard.weak_shard(world, rank, g.n, 2)
    else:
        r_total = 3
        begin, count = shard.strong_shard(world, rank, g.n * r_total - 5)
    ids = np.arange(begin, begin + count)
    rows = oracle.walk(g.row_ptr, g.col, None, starts, l, p, q, seed, ids)
    # gather (variable sizes: pad to the largest share)
    n = torch.tensor([count])
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    mx = int(max(s.item() for s in sizes))
    buf = torch.full((mx, l), -9, dtype=torch.int32)
    buf[:count] = torch.from_numpy(rows)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    # the timed region is the slowest rank's
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        whole = np.concatenate([p[: int(s.item())].numpy() for p, s in zip(parts, sizes)])
        total = world * g.n * 2 if mode == "weak" else g.n * r_total - 5
        want = oracle.walk(g.row_ptr, g.col, None, starts, l, p, q, seed, np.arange(total))
        out_q.put((bool(np.array_equal(whole, want)), float(t.item()), whole.shape[0]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_rank_shards_equal_one_process(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    ok, tmax, n = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert ok and tmax == 2.0 and n > 0


def test_shard_arithmetic():
    for world in (1, 2, 3, 8):
        spans = [shard.strong_shard(world, k, 1001) for k in range(world)]
        assert spans[0][0] == 0 and sum(c for _, c in spans) == 1001
        assert all(a + c == b for (a, c), (b, _) in zip(spans, spans[1:]))
        assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
        w = [shard.weak_shard(world, k, 100, 3) for k in range(world)]
        assert all(rt == 3 * world for rt, _, _ in w)
        assert [b for _, b, _ in w] == [300 * k for k in range(world)]
    with pytest.raises(ValueError):
        shard.weak_shard(2, 2, 10, 1)
