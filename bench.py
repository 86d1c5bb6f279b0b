#!/usr/bin/env python3
"""Benchmark of the GB300 node2vec walk sampler.

Metric: node2vec walk steps/s (real transitions, i.e. written entries != -1)
and the fraction of the HBM roofline, bit-exact to the CPU oracle, for the
persistent degree-binned sampler beside the plain one-thread-per-walker,
one-launch-per-step sampler.

A "step" of this benchmark is one pass of the whole hot path over one batch:
every walk of the workload (r walks from every vertex, length l) for every
(p, q) setting of the workload, on a resident graph, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat26]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

Under torchrun (N > 1) every rank runs the same per-GPU workload on its own
range of walk ids (weak scaling, no collective on the data path); the timed
region is bracketed by barriers and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

REPO = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, REPO)

METRIC = "node2vec walk steps/sec + % HBM roofline, bit-exact; persistent vs plain kernel"
UNIT = "steps/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--variant", default="persistent", choices=["persistent", "binned", "plain"])
    ap.add_argument("--compare", default="plain,binned,stored",
                    help="variants timed once beside the main one (stored: the stored-table baseline)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle baseline leg")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--tune", default="", help="JSON dict of n2v_tune fields")
    ap.add_argument("--pq", default="", help="override (p,q) list, e.g. '1,1;0.25,4'")
    ap.add_argument("--r", type=int, default=0, help="override walks per vertex")
    ap.add_argument("--walk-count", type=int, default=0, help="limit walks per launch (profiling cases)")
    ap.add_argument("--shuffle-starts", type=int, default=0,
                    help="start vertices in a seeded random order, so that --walk-count walks start at a uniform "
                         "sample of the vertices (profiling cases; without it R-MAT's first ids are its hubs)")
    ap.add_argument("--compare-rounds", type=int, default=1,
                    help="the compared variants run the first R rounds (every start vertex R times)")
    ap.add_argument("--compare-walks", type=int, default=0,
                    help="cap on the walks of the compared variants (0: the workload's default)")
    ap.add_argument("--c2", type=int, default=-1,
                    help="add the R-MAT 20 persistent / binned / plain block (-1: per workload)")
    ap.add_argument("--sweep", default="", help="run every workload of a sweep (skew, wec), one JSON line each")
    ap.add_argument("--ingest-ncu", nargs=2, metavar=("LAUNCH_CSV", "BENCH_JSON"), default=None,
                    help="write profiles/traffic_<variant>_<workload>.json from an ncu launch list (with DRAM bytes) "
                         "of a bench run with --no-cpu --no-e2e, and that run's JSON line")
    ap.add_argument("--cuda-graph", type=int, default=-1, help="record the launches as a CUDA graph (-1: per workload)")
    ap.add_argument("--autotune", type=int, default=1, help="tune the persistent sampler on a sample first")
    ap.add_argument("--tune-cache", default="",
                    help="directory of stored autotuner results: reuse the one for this graph, GPU, build and "
                         "sample instead of tuning again (stored after a miss)")
    ap.add_argument("--jobs", type=int, default=10_000, help="serving workload: number of jobs")
    ap.add_argument("--load", type=float, default=0.8, help="serving: arrival rate as a fraction of capacity")
    return ap.parse_args()


# workload-specific defaults: the scale-26 graph runs in 8M-walker launches
# (FN-Multi-style rounds) recorded as one CUDA graph; its compared variants run
# 2^19 walks in four ranges spread over the job; its end-to-end leg streams the
# rows to host memory chunk by chunk; and the line carries the R-MAT 20
# persistent / binned / plain block.  Where hub caches are loaded (the sizes
# given here), the autotuner measures them and picks how much of them to use.
WORKLOAD_DEFAULTS = {
    "rmat26": {"tune": {"chunk_walkers": 1 << 23}, "cuda_graph": 1, "compare_walks": 1 << 19, "compare_ranges": 4,
               "c2": 1, "e2e_stream": 1},
    # R-MAT 22 is the profiling case; its hub caches (top 0.1%, 64 bitmaps) are loaded so that
    # runs with --tune can switch them on
    "rmat22": {"tune": {"bitmap_hubs": 64, "hub_count": 4194, "hub_budget_mb": 2048}, "cuda_graph": 1},
    # the hub cache of the top 0.1% of vertices (2^23 / 1000 hashed sets) and 32 rank bitmaps;
    # the autotuner picks how many of each to keep
    "rmat23w": {"tune": {"hub_count": 8388, "hub_budget_mb": 8192, "bitmap_hubs": 32}},
    "rmat20": {"tune": {"bitmap_hubs": 32}},
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# the sources the sampler kernels are compiled from (the autotuner, serving
# loop, graph loader and the header's documentation are not part of them)
KERNEL_SOURCES = ["paper_1805_00280_gb300/csrc/n2v_walk.cu", "paper_1805_00280_gb300/csrc/n2v_step.cuh",
                  "paper_1805_00280_gb300/csrc/n2v_internal.cuh"]


def csrc_digest() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(REPO, f), "rb").read())
    return h.hexdigest()[:16]


def workload_params(args):
    from paper_1805_00280_gb300 import graphs as G

    wl = G.WORKLOADS[args.workload]
    pq = list(wl.pq)
    if args.pq:
        pq = [tuple(float(x) for x in s.split(",")) for s in args.pq.split(";")]
    r = args.r or wl.r
    return wl, pq, r


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peak_hbm():
    p = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(workload: str, variant: str, tune: dict):
    """Per-launch DRAM bytes from a committed ncu summary of this workload and variant, if the kernel
    sources have not changed since; with whether the run's tuning is the one it was captured with."""
    p = os.path.join(REPO, "profiles", f"traffic_{variant}_{workload}.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None, None
    if d.get("csrc_sha") != csrc_digest():
        return None, None
    return d.get("dram_bytes_per_launch"), effective_tune(d.get("tune")) == effective_tune(tune)


def dram_fraction(dram_bytes_per_call, mean_call_ms: list, peak_gbs: float) -> dict | None:
    """Measured DRAM bytes of one call (from an ncu capture) over the mean call time of this run:
    the achieved DRAM bandwidth and its fraction of the peak (None without a capture)."""
    if not dram_bytes_per_call or not mean_call_ms or sum(mean_call_ms) <= 0:
        return None
    gbs = dram_bytes_per_call * len(mean_call_ms) / (sum(mean_call_ms) / 1e3) / 1e9
    return {"achieved": gbs, "unit": "GB/s", "frac": gbs / peak_gbs}


def effective_tune(tune: dict | None) -> dict | None:
    """The tuning as the persistent sampler runs it: blocks_per_sm 0 means its default of 20
    resident warps per SM, i.e. five 128-thread blocks."""
    if tune is None:
        return None
    t = dict(tune)
    if t.get("blocks_per_sm", 0) <= 0:
        t["blocks_per_sm"] = 5
    return t


# --------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on a bounded sample of walk ids

def oracle_mod():
    """The CPU oracle (test infrastructure; only the CPU-baseline and parity legs use it)."""
    import oracle

    return oracle


def cpu_oracle_sample(g, starts_np, r, l, pq, seed, budget_s, threads, id_space, rng_seed=0, check=None):
    import numpy as np

    import oracle

    rng = np.random.default_rng(rng_seed)
    n_ids = 256
    done_steps, done_time, sample_desc, parity_ok, parity_rows = 0, 0.0, [], True, 0
    t_start = time.perf_counter()
    while True:
        ids = np.sort(rng.choice(id_space, size=min(n_ids, id_space), replace=False))
        for (p, q) in pq:
            t0 = time.perf_counter()
            rows = oracle.walk(g.row_ptr, g.col, g.w, starts_np, l, p, q, seed, ids, threads=threads)
            dt = time.perf_counter() - t0
            done_time += dt
            done_steps += int((rows >= 0).sum())
            if check is not None:
                ok = check(p, q, ids, rows)
                parity_ok &= ok
                parity_rows += len(ids)
        sample_desc.append(len(ids))
        elapsed = time.perf_counter() - t_start
        if elapsed > budget_s * 0.5 or n_ids >= id_space:
            break
        n_ids = min(id_space, int(n_ids * max(2.0, min(8.0, budget_s * 0.5 / max(elapsed, 1e-3)))))
    return done_steps, done_time, sample_desc, parity_ok, parity_rows


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    from paper_1805_00280_gb300 import graphs as G

    wl, pq, r = workload_params(args)
    g = G.workload_graph(wl.name)
    starts = np.arange(g.n, dtype=np.int32)
    threads = os.cpu_count() or 1
    if not pq:  # serving workload: the oracle on the first jobs of the same mix
        import oracle

        jobs = serving_jobs(g.n, min(args.jobs, 64))
        t0, st, used = time.perf_counter(), 0, 0
        for jb in jobs:
            s_np = G.uniform(jb["seed"], jb["stream"], g.n, jb["size"]).astype(np.int32)
            ids = np.arange(min(jb["size"], 2048))
            rows = oracle.walk(g.row_ptr, g.col, g.w, s_np, jb["l"], jb["p"], jb["q"], jb["seed"], ids, threads=threads)
            st += int((rows >= 0).sum())
            used += 1
            if time.perf_counter() - t0 > 60:
                break
        dt = time.perf_counter() - t0
        value = st / dt
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                          "config": {"workload": wl.name, "jobs_sampled": used},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                           "sample": f"first 2048 walks of each of the first {used} jobs"},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    per_step_budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    # size the per-step sample once
    steps_done, t_done, desc, _, _ = cpu_oracle_sample(g, starts, r, wl.l, pq, wl.seed, per_step_budget, threads,
                                                      g.n * r)
    n_ids = desc[-1]
    rng = np.random.default_rng(5)
    import oracle

    times, steps = [], []
    for s in range(args.warmup + args.steps):
        ids = np.sort(rng.choice(g.n * r, size=n_ids, replace=False))
        t0 = time.perf_counter()
        st = 0
        for (p, q) in pq:
            rows = oracle.walk(g.row_ptr, g.col, g.w, starts, wl.l, p, q, wl.seed, ids, threads=threads)
            st += int((rows >= 0).sum())
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            steps.append(st)
    value = sum(steps) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "n": g.n, "nnz": g.nnz, "r": r, "l": wl.l, "pq": pq,
                   "sample_walks_per_pq_per_step": n_ids},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_ids} random walk ids per (p,q) per step of {g.n * r}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    from paper_1805_00280_gb300 import graphs as G
    from paper_1805_00280_gb300 import n2v

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    wl, pq, r = workload_params(args)
    wdef = WORKLOAD_DEFAULTS.get(wl.name, {})
    t0 = time.perf_counter()
    g = G.workload_graph(wl.name)
    gen_s = time.perf_counter() - t0
    tune_kw = dict(wdef.get("tune", {}))
    tune_kw.update(json.loads(args.tune) if args.tune else {})
    tune = n2v.default_tune(**tune_kw)
    cuda_graph = bool(wdef.get("cuda_graph", 0)) if args.cuda_graph < 0 else bool(args.cuda_graph)
    stream = torch.cuda.Stream(dev)  # a side stream: CUDA graphs cannot record the legacy stream
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    graph = n2v.Graph.from_csr(g, tune=tune, device=dev)
    load_s = time.perf_counter() - t0
    tuned = None
    if args.autotune and args.variant == "persistent":
        t0 = time.perf_counter()
        # the job's first walks (walk id i starts at vertex i mod n): the whole job when it
        # has at most 2^20 walks, else 2^20 walks of 20 steps, which fill every resident warp
        # many times over
        n_job = g.n * wl.r
        n_tune = min(1 << 20, n_job)
        # the whole job when it has at most 2^20 walks; else 2^20 start vertices drawn at random
        # (R-MAT's first ids are its hubs: a prefix of the job would over-sample them)
        tune_starts = np.resize(np.arange(g.n, dtype=np.int32), n_tune) if n_tune == n_job else \
            np.arange(g.n, dtype=np.int32)
        l_tune = wl.l if n_tune == n_job else min(wl.l, 20)
        from_cache = None
        if args.tune_cache:
            from paper_1805_00280_gb300 import tune_cache

            best, ms, from_cache = tune_cache.autotune_cached(tune_cache.TuneCache(args.tune_cache), graph, g,
                                                              tune_starts, l_tune, pq[0][0], pq[0][1], wl.seed,
                                                              sample=n_tune, stream=stream)
        else:
            best, ms = n2v.autotune(graph, tune_starts, l_tune, pq[0][0], pq[0][1], wl.seed, sample=n_tune,
                                    stream=stream)
        tuned = {"tune": best.as_dict(), "sample_ms": round(ms, 3), "tune_s": round(time.perf_counter() - t0, 2)}
        if from_cache is not None:
            tuned["cache"] = "hit" if from_cache else "miss"
        tune = best
    caches = None
    if args.variant == "persistent":
        caches = cache_ab(n2v, graph, tune, g, wl.l, pq[0][0], pq[0][1], wl.seed, stream, dev)
    info = graph.info()
    l = wl.l
    n_start = g.n
    from paper_1805_00280_gb300 import shard

    r_total, walk_begin, W = shard.weak_shard(world, rank, n_start, r)  # rank k runs rounds [k r, (k+1) r)
    if args.walk_count:
        W = min(W, args.walk_count)
    starts_np = np.arange(n_start, dtype=np.int32)
    if args.shuffle_starts:
        starts_np = np.random.default_rng(args.shuffle_starts).permutation(n_start).astype(np.int32)
    starts = torch.from_numpy(starts_np).to(dev)
    outs = [torch.empty((W, l), dtype=torch.int32, device=dev) for _ in pq]
    variant = n2v.VARIANTS[args.variant] | (n2v.N2V_FLAG_CUDA_GRAPH if cuda_graph else 0)
    ws_bytes = max(n2v.n2v_walk_ws_bytes(graph.handle, W, l, variant), 256)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.int64, device=dev)
    flush = torch.empty(max(args.flush_mb, 1) * (1 << 20) // 4, dtype=torch.int32, device=dev)

    def launch(i, v=variant, out=None):
        p, q = pq[i]
        n2v.n2v_walk(graph.handle, starts, n_start, r_total, l, p, q, wl.seed, walk_begin, W,
                     outs[i] if out is None else out, ws, v, stream)

    for _ in range(args.warmup):
        for i in range(len(pq)):
            launch(i)
    torch.cuda.synchronize(dev)
    st = n2v.n2v_stream_status(graph.handle, stream)
    if st != n2v.N2V_OK:
        raise RuntimeError(f"sampler status {n2v.n2v_strerror(st)}")

    if n2v.stats_build():
        n2v.n2v_step_stats(reset=True)  # the stats build counts the timed steps only
    # ---- timed region: K steps, each = every (p,q) job of the workload
    clocks = ClockSampler(local)
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in pq]
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s)  # evict L2 (129 MB) between steps; outside the events
        for i in range(len(pq)):
            evs[s][i][0].record(stream)
            launch(i)
            evs[s][i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    launch_ms = [[a.elapsed_time(b) for (a, b) in row] for row in evs]
    total_ms = sum(sum(row) for row in launch_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    st = n2v.n2v_stream_status(graph.handle, stream)
    if st != n2v.N2V_OK:
        raise RuntimeError(f"sampler status {n2v.n2v_strerror(st)}")
    step_stats = n2v.n2v_step_stats(reset=True) if n2v.stats_build() else None

    # ---- work done per step (deterministic rows, so the same every step)
    trans, abytes, lbytes = [], [], []
    for i in range(len(pq)):
        tr, by, lo = n2v.traffic(graph, starts, walk_begin, outs[i])
        trans.append(tr)
        abytes.append(by)
        lbytes.append(lo)
    steps_per_step = sum(trans) * world  # all ranks
    value = steps_per_step * args.steps / (total_ms / 1e3)
    mean_launch_ms = [statistics.mean(launch_ms[s][i] for s in range(args.steps)) for i in range(len(pq))]

    # ---- roofline of the dominant kernel (the persistent sampler: one launch per (p,q))
    peak, peak_kind = measured_peak_hbm()
    achieved = sum(abytes) / (sum(mean_launch_ms) / 1e3) / 1e9
    dram, dram_same_tune = ncu_traffic(wl.name, args.variant, tune.as_dict())
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": dram, "traffic_same_tuning": dram_same_tune,
                "traffic_source": f"profiles/traffic_{args.variant}_{wl.name}.json" if dram else None,
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": [int(b) for b in abytes],
                "kernel": {"persistent": "k_persistent", "binned": "k_binned_step", "plain": "k_plain_step"}[args.variant],
                "bytes_model": "16 + 4 deg(v) (1+weighted) + [k>=1](16 + 4 deg(t)) + 4 per real transition"}
    # what the committed ncu capture's DRAM bytes come to over this run's call times
    roofline["dram"] = dram_fraction(dram, mean_launch_ms, peak)
    # the conservative lower model: N(v) and the output only, no N(t) message
    lower_achieved = sum(lbytes) / (sum(mean_launch_ms) / 1e3) / 1e9
    roofline["lower_model"] = {"bytes_model": "16 + 4 deg(v) (1+weighted) + 4 per real transition",
                               "algorithmic_bytes_per_launch": [int(b) for b in lbytes],
                               "achieved": lower_achieved, "frac": lower_achieved / peak}
    step_ms = [sum(row) for row in launch_ms]

    # ---- the other variants, once each, beside the main variant on the same rows: the first
    #      `compare_rounds` rounds of walk ids, or (large jobs) contiguous id ranges spread
    #      evenly over the job
    compare = {}
    ranges = compare_ranges(W, n_start, args, wdef)
    names = [v for v in args.compare.split(",") if v in ("plain", "binned", "persistent") and v != args.variant]
    if names:
        compare = compare_variants(n2v, graph, starts, n_start, r_total, l, pq, wl.seed, walk_begin, ranges,
                                   [args.variant] + names, outs, ws, stream, dev, world, flush, args.variant)
    if "stored" in args.compare.split(","):
        Wc = ranges[0][1]  # the first range starts at walk id offset 0
        compare["stored"] = stored_compare(n2v, graph, g, starts, n_start, r_total, l, pq, wl.seed, walk_begin,
                                           Wc, outs, stream, dev, world, flush)
        compare["stored"]["walks_per_pq"] = Wc

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        starts_h = torch.from_numpy(starts_np).pin_memory()
        out_h = torch.empty((W, l), dtype=torch.int32).pin_memory()
        starts_d = torch.empty_like(starts)
        K2 = max(1, min(args.steps, 3))
        streamed = bool(wdef.get("e2e_stream", 0)) and tune.chunk_walkers > 0 and tune.chunk_walkers < W
        if streamed:
            # FN-Multi-style output: chunks of chunk_walkers walks into a two-slot device ring, each
            # chunk copied to the host on a second stream while the next one runs
            ring_walks = tune.chunk_walkers
            ring = torch.empty((2, ring_walks, l), dtype=torch.int32, device=dev)
            copy_stream = torch.cuda.Stream(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        a.record(stream)
        for s in range(K2):
            for i in range(len(pq)):
                starts_d.copy_(starts_h, non_blocking=True)
                p, q = pq[i]
                if streamed:
                    n2v.n2v_walk_stream(graph.handle, starts_d, n_start, r_total, l, p, q, wl.seed, walk_begin, W,
                                        out_h, ring, ring_walks, 2, ws, n2v.VARIANTS[args.variant], stream,
                                        copy_stream)
                else:
                    n2v.n2v_walk(graph.handle, starts_d, n_start, r_total, l, p, q, wl.seed, walk_begin, W, outs[i],
                                 ws, variant, stream)
                    out_h.copy_(outs[i], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = a.elapsed_time(b)
        if world > 1:
            t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        path = ("pinned host starts -> n2v_walk_stream (chunks of %d walks, 2-slot device ring, each chunk copied "
                "to pinned host walks while the next runs), per (p,q)" % ring_walks if streamed else
                "pinned host starts -> n2v_walk -> pinned host walks, per (p,q)")
        e2e = {"value": steps_per_step * K2 / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": 4 * n_start * len(pq), "d2h_bytes_per_step": 4 * W * l * len(pq),
               "steps": K2, "path": path}
        # SHA-256 of every (p,q) job's full output, through the host buffer (after the timing); the
        # streamed rows must equal the timed device output
        out_sha = []
        same = True
        for i in range(len(pq)):
            if streamed:
                p, q = pq[i]
                n2v.n2v_walk_stream(graph.handle, starts_d, n_start, r_total, l, p, q, wl.seed, walk_begin, W, out_h,
                                    ring, ring_walks, 2, ws, n2v.VARIANTS[args.variant], stream, copy_stream)
                torch.cuda.synchronize(dev)
                for c0 in range(0, W, 1 << 22):
                    same &= bool(torch.equal(out_h[c0:c0 + (1 << 22)].to(dev, non_blocking=False),
                                             outs[i][c0:c0 + (1 << 22)]))
            else:
                out_h.copy_(outs[i])
            out_sha.append(hashlib.sha256(out_h.numpy()).hexdigest())
        e2e["output_sha256"] = out_sha
        if streamed:
            e2e["streamed_rows_equal_device_rows"] = same
            del ring
        del out_h

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        out_np_cache = {}

        def check(p, q, ids, rows):
            i = pq.index((p, q))
            got = outs[i][torch.from_numpy(ids).to(dev)].cpu().numpy()
            return bool(np.array_equal(got, rows))

        steps_c, t_c, desc, ok, nrows = cpu_oracle_sample(g, starts_np, r, l, pq, wl.seed, args.cpu_seconds, threads,
                                                          W, check=check)
        cpu = {"value": steps_c / t_c, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"random walk-id samples of sizes {desc} per (p,q) out of {W}"}
        # the same oracle on one core, on a small sample of the first job
        ids1 = np.sort(np.random.default_rng(2).choice(W, size=min(256, W), replace=False))
        t0 = time.perf_counter()
        rows1 = oracle_mod().walk(g.row_ptr, g.col, g.w, starts_np, l, pq[0][0], pq[0][1], wl.seed, ids1, threads=1)
        cpu["one_core"] = {"value": int((rows1 >= 0).sum()) / (time.perf_counter() - t0), "unit": UNIT,
                           "sample": f"{len(ids1)} random walk ids of the first (p,q)"}
        ok &= check(pq[0][0], pq[0][1], ids1, rows1)
        # parity beyond the timed sample: at least 2^14 random walk ids in all, and every walk
        # that starts at one of the 100 highest-degree vertices
        n_rand = sum(desc)
        extra = np.sort(np.random.default_rng(3).choice(W, size=min(max(0, (1 << 14) - n_rand), W), replace=False))
        hubs = np.sort(np.argsort(g.degrees(), kind="stable")[-100:])
        slot_of = np.argsort(starts_np)  # index i of vertex h in starts: walk ids k n + i start at h
        hub_ids = np.sort(np.array([k * n_start + slot_of[h] for k in range(max(1, W // n_start)) for h in hubs],
                                   dtype=np.int64))
        hub_ids = hub_ids[hub_ids < W]
        for ids_x in (extra, hub_ids):
            if ids_x.size == 0:
                continue
            for (p, q) in pq:
                rows_x = oracle_mod().walk(g.row_ptr, g.col, g.w, starts_np, l, p, q, wl.seed, ids_x, threads=threads)
                ok &= check(p, q, ids_x, rows_x)
                nrows += len(ids_x)
        parity = {"oracle_rows_checked": nrows + len(ids1), "random_walk_ids": n_rand + int(extra.size),
                  "hub_start_walk_ids": int(hub_ids.size), "hub_vertices": int(hubs.size), "bit_exact": ok}

    # ---- the R-MAT 20 workload's three samplers on the same rows (single-GPU runs)
    c2 = None
    use_c2 = bool(wdef.get("c2", 0)) if args.c2 < 0 else bool(args.c2)
    if use_c2 and world == 1 and args.variant == "persistent":
        c2 = c2_block(n2v, dev, stream, flush, check_oracle=not args.no_cpu)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "ms_per_step_median": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "desc": wl.note, "n": g.n, "nnz": g.nnz, "weighted": g.w is not None,
                   "r": r, "l": l, "pq": pq, "walks_per_gpu": W, "variant": args.variant,
                   "tune": tune.as_dict(), "autotune": tuned, "cuda_graph": cuda_graph,
                   "hubs": info.hub_count, "hub_min_degree": info.hub_min_degree,
                   "max_degree": info.max_degree,
                   "l2": f"flushed between steps ({args.flush_mb} MB write); output {4 * W * l * len(pq) >> 20} MB",
                   "gen_s": round(gen_s, 2), "load_s": round(load_s, 3),
                   "start_order": f"seeded permutation {args.shuffle_starts}" if args.shuffle_starts else "vertex id"},
        "walks_per_s": W * len(pq) * world * args.steps / (total_ms / 1e3),
        "nominal_steps_per_s": W * l * len(pq) * world * args.steps / (total_ms / 1e3),
        "real_transitions_per_step": steps_per_step,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * len(pq) * (
            (-(-W // tune.chunk_walkers) if tune.chunk_walkers > 0 else 1) if args.variant == "persistent" else l),
        "clocks": clk,
        "compare": compare,
        "hub_caches": caches,
        "c2": c2,
        "parity": parity,
        "wall_s_timed": wall,
    }
    if step_stats is not None:
        line["step_stats"] = step_stats
        line["build"] = "stats (per-step counters on: timings are not bench values)"
    if args.sweep:
        line["sweep"] = args.sweep
        line["degree_bins"] = degree_bins(graph, info, outs[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    graph.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------
# serving: continuous batching of walk jobs with Poisson arrivals

def serving_jobs(n_vertices: int, count: int, run_seed: int = 1):
    """The job mix: start-set size log-uniform in [1, 2^20] (uniform vertices, with
    replacement), l uniform in {10, 20, 40, 80}, p and q log-uniform in [0.25, 4]
    quantised to Q16, seed = hash(run seed, job id)."""
    import numpy as np

    from paper_1805_00280_gb300 import graphs as G

    raw = G.raw64(run_seed, 77, 4 * count).reshape(count, 4)
    u = (raw >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    jobs = []
    for j in range(count):
        size = max(1, min(1 << 20, int(np.exp(u[j, 0] * np.log(1 << 20)))))
        l = [10, 20, 40, 80][int(raw[j, 1] % np.uint64(4))]
        p = round(float(np.exp(np.log(0.25) + u[j, 2] * np.log(16.0))) * 65536) / 65536
        q = round(float(np.exp(np.log(0.25) + u[j, 3] * np.log(16.0))) * 65536) / 65536
        jobs.append({"size": size, "l": l, "p": p, "q": q, "seed": int(G.raw64(run_seed, 1000 + j, 1)[0]),
                     "stream": 5000 + j})
    return jobs


def run_serving(args):
    import numpy as np
    import torch

    from paper_1805_00280_gb300 import graphs as G
    from paper_1805_00280_gb300 import n2v

    rank, world, local = dist_env()
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    wl = G.WORKLOADS[args.workload]
    t0 = time.perf_counter()
    g = G.workload_graph(wl.name)
    gen_s = time.perf_counter() - t0
    graph = n2v.Graph.from_csr(g, device=dev)
    best, _ = n2v.autotune(graph, np.arange(g.n, dtype=np.int32), 20, 1.0, 1.0, 1, sample=min(1 << 20, g.n),
                           stream=stream)
    jobs = serving_jobs(g.n, args.jobs)
    for jb in jobs:
        jb["starts"] = G.uniform(jb["seed"], jb["stream"], g.n, jb["size"]).astype(np.int32)
    free, total = torch.cuda.mem_get_info(dev)
    arena_bytes = int(min(free * 0.6, 96 << 30))  # admission by free HBM: the arena is what is free
    cfg = n2v.n2v_serve_cfg_default()
    srv = n2v.Server(graph, arena_bytes, cfg, stream)
    counted = torch.zeros((), dtype=torch.int64, device=dev)

    copy_stream = torch.cuda.Stream(dev)
    kept = {}  # job index -> host copy of its rows in the mix (the parity sample)

    def run_batch(sel, arrivals=None, keep_every=0):
        """Serve jobs `sel`; arrivals[i] = submit time offset (None: all at t=0).  With keep_every,
        the rows of every keep_every-th job are copied to the host (on a side stream) before release.
        Returns (makespan_s, latencies_s, real transitions)."""
        counted.zero_()
        sub_t, lat = {}, []
        jid_to_job = {}
        pending = sorted(range(len(sel)), key=lambda i: 0.0 if arrivals is None else arrivals[i])
        pi = 0
        t_start = time.perf_counter()
        done = 0
        while done < len(sel):
            now = time.perf_counter() - t_start
            while pi < len(pending) and (arrivals is None or arrivals[pending[pi]] <= now):
                jb = jobs[sel[pending[pi]]]
                jid = srv.submit(jb["starts"], jb["l"], jb["p"], jb["q"], jb["seed"])
                sub_t[jid] = t_start + (0.0 if arrivals is None else arrivals[pending[pi]])
                jid_to_job[jid] = sel[pending[pi]]
                pi += 1
            srv.step()
            for jid in srv.poll():
                lat.append(time.perf_counter() - sub_t[jid])
                counted.add_((srv.rows(jid) >= 0).sum())
                jx = jid_to_job[jid]
                if keep_every and jx % keep_every == 0:
                    with torch.cuda.stream(copy_stream):  # the job is complete: copy beside the running ticks
                        kept[jx] = srv.rows(jid).to("cpu", non_blocking=True)
                    copy_stream.synchronize()
                srv.release(jid)
                done += 1
            if pi < len(pending) and arrivals is not None:
                time.sleep(0.0002)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t_start, lat, int(counted.item())

    # capacity: a batch of jobs submitted at once, back to back
    cap_sel = list(range(min(len(jobs), 300)))
    run_batch(cap_sel[:20])  # warm-up
    span, _, steps = run_batch(cap_sel)
    capacity = steps / span                                # steps/s
    mean_steps = steps / len(cap_sel)                      # steps per job (this mix)
    rate = args.load * capacity / mean_steps               # jobs/s
    rng = np.random.default_rng(11)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(jobs)))
    clocks = ClockSampler(local)
    ticks0 = srv.stats()["ticks"]
    clocks.start()
    span, lat, steps = run_batch(list(range(len(jobs))), arrivals, keep_every=max(1, len(jobs) // 100))
    clk = clocks.stop()
    ticks = srv.stats()["ticks"] - ticks0
    st = n2v.n2v_stream_status(graph.handle, stream)
    if st != n2v.N2V_OK:
        raise RuntimeError(n2v.n2v_strerror(st))
    # parity of the sampled jobs: the rows each had in the mix equal the same job alone (n2v_walk),
    # and sampled rows of each equal the oracle's
    same_alone, oracle_ok, oracle_rows = True, True, 0
    rng_p = np.random.default_rng(55)
    for jx, rows_mix in sorted(kept.items()):
        jb = jobs[jx]
        alone = n2v.walk(graph, jb["starts"], 1, jb["l"], jb["p"], jb["q"], jb["seed"], "persistent", stream=stream)
        torch.cuda.synchronize(dev)
        same_alone &= bool(torch.equal(alone.cpu(), rows_mix))
        if not args.no_cpu:
            sel = np.sort(rng_p.choice(jb["size"], size=min(32, jb["size"]), replace=False))
            want = oracle_mod().walk(g.row_ptr, g.col, None, jb["starts"], jb["l"], jb["p"], jb["q"], jb["seed"], sel,
                                     threads=os.cpu_count() or 1)
            oracle_ok &= bool(np.array_equal(rows_mix.numpy()[sel], want))
            oracle_rows += len(sel)
        del alone
    parity = {"jobs_checked": len(kept), "mix_equals_alone": same_alone,
              "oracle_rows_checked": oracle_rows, "bit_exact": oracle_ok and same_alone}
    st = n2v.n2v_stream_status(graph.handle, stream)
    if st != n2v.N2V_OK:
        raise RuntimeError(n2v.n2v_strerror(st))
    # the jobs one at a time through the plain sampler (a bounded subset)
    seq_sel = list(range(min(len(jobs), 40)))
    seq_steps, seq_ms, seq_lat = 0, 0.0, []
    for i in seq_sel:
        jb = jobs[i]
        s_d = torch.from_numpy(jb["starts"]).to(dev)
        out = torch.empty((jb["size"], jb["l"]), dtype=torch.int32, device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n2v.n2v_walk(graph.handle, s_d, jb["size"], 1, jb["l"], jb["p"], jb["q"], jb["seed"], 0, jb["size"], out, None,
                     n2v.N2V_PLAIN, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms += a.elapsed_time(b)
        seq_lat.append(a.elapsed_time(b) / 1e3)
        seq_steps += int((out >= 0).sum())
    srv.close()
    lat = np.array(lat)
    line = {
        "metric": METRIC, "value": steps / span, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "desc": "serving on R-MAT scale 24, ef 16", "n": g.n, "nnz": g.nnz,
                   "jobs": len(jobs), "job_size": "log-uniform in [1, 2^20] uniform starts, with replacement",
                   "l": [10, 20, 40, 80], "pq": "log-uniform [0.25, 4], Q16", "arrivals": "Poisson",
                   "load": args.load, "arena_bytes": arena_bytes, "tick_walkers": cfg.tick_walkers,
                   "tune": best.as_dict(), "gen_s": round(gen_s, 2)},
        "serving": {"throughput_steps_per_s": steps / span, "jobs_per_s": len(jobs) / span,
                    "capacity_steps_per_s": capacity, "arrival_rate_jobs_per_s": rate,
                    "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                    "latency_mean_s": float(lat.mean()), "makespan_s": span, "real_transitions": steps,
                    "latency_to": "rows resident in HBM (job polled complete)"},
        "sequential_plain": {"jobs": len(seq_sel), "value": seq_steps / (seq_ms / 1e3), "unit": UNIT,
                             "service_time_p50_s": float(np.percentile(seq_lat, 50)),
                             "note": "the first jobs one at a time through the plain sampler, no queueing"},
        "gpu_launches": int(ticks),
        "clocks": clk,
        "parity": parity,
    }
    line["speedup_over_sequential_plain"] = line["value"] / line["sequential_plain"]["value"]
    print(json.dumps(line), flush=True)


def degree_bins(graph, info, rows) -> dict:
    """Vertices and walk visits per degree bin ([0]: degree 0, [i]: [2^(i-1), 2^i)), as in the
    degree-vs-frequency view of Section 3.3: how often the walks stand on vertices of each degree."""
    import torch

    rp = graph.row_ptr
    visits = torch.zeros(34, dtype=torch.int64, device=rp.device)
    flat = rows.reshape(-1)
    for c0 in range(0, flat.numel(), 1 << 26):
        v = flat[c0:c0 + (1 << 26)].to(torch.int64)
        v = v[v >= 0]
        d = rp[v + 1] - rp[v]
        b = torch.where(d > 0, torch.floor(torch.log2(d.clamp(min=1).to(torch.float64))).to(torch.int64) + 1,
                        torch.zeros_like(d))
        visits += torch.bincount(b, minlength=34)[:34]
    vs = [int(x) for x in info.deg_hist]
    last = max([i for i in range(34) if vs[i]] + [0]) + 1
    return {"vertices": vs[:last], "visits": [int(x) for x in visits.cpu()][:last]}


def cache_ab(n2v, graph, tune, g, l: int, p: float, q: float, seed: int, stream, dev) -> dict | None:
    """The hub caches the graph was loaded with, each switched on over the chosen tuning and timed
    on the autotuner's kind of sample (2^20 random start vertices, walks of up to 20 steps): the
    measured evidence behind the tuner's choice.  None when no cache was loaded."""
    import numpy as np
    import torch

    loaded = graph.tune_loaded
    if loaded.hub_count <= 0 and loaded.bitmap_hubs <= 0:
        return None
    rng = np.random.default_rng(9)
    sample = min(1 << 20, g.n)
    starts = torch.from_numpy(rng.choice(g.n, size=sample, replace=False).astype(np.int32)).to(dev)
    ls = min(l, 20)
    out = torch.empty((sample, ls), dtype=torch.int32, device=dev)
    base = tune.as_dict()
    cands = [("chosen", {})]
    if loaded.hub_count > 0:
        cands.append(("hashed_sets", {"hub_count": loaded.hub_count, "hub_budget_mb": loaded.hub_budget_mb}))
    if loaded.bitmap_hubs > 0:
        cands.append(("rank_bitmaps", {"bitmap_hubs": loaded.bitmap_hubs}))
    if loaded.hub_count > 0 and loaded.bitmap_hubs > 0:
        cands.append(("both", {"hub_count": loaded.hub_count, "hub_budget_mb": loaded.hub_budget_mb,
                               "bitmap_hubs": loaded.bitmap_hubs}))
    res = {}
    for name, over in cands:
        t = n2v.default_tune(**{**base, **over})
        graph.retune(t, stream)
        info = graph.info()
        n2v.walk(graph, starts, 1, ls, p, q, seed, "persistent", out=out, stream=stream)  # warm-up
        best = None
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            n2v.walk(graph, starts, 1, ls, p, q, seed, "persistent", out=out, stream=stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
        res[name] = {"ms": round(best, 3), "hub_count": info.hub_count, "bitmap_hubs": info.bitmap_hubs}
    graph.retune(tune, stream)
    return {"sample_walks": sample, "l": ls, "candidates": res}


def compare_ranges(W: int, n_start: int, args, wdef: dict) -> list[tuple[int, int]]:
    """Walk-id ranges (offset, count) inside this rank's W walks on which the compared variants run.

    Small jobs: the first `compare_rounds` rounds (every start vertex that many times), capped by
    `compare_walks`.  Jobs with a per-workload `compare_ranges` default: that many contiguous
    ranges of compare_walks / ranges walks each, at evenly spaced offsets over the job, so that
    both the low-numbered hubs of an R-MAT graph and its sparse tail are sampled."""
    k = int(wdef.get("compare_ranges", 1))
    total = min(W, args.compare_walks if args.compare_walks > 0 else int(wdef.get("compare_walks", 1 << 22)))
    if k <= 1:
        return [(0, min(total, n_start * max(1, args.compare_rounds)))]
    each = max(1, total // k)
    return [(min(i * (W // k), W - each), each) for i in range(k)]


def compare_variants(n2v, graph, starts, n_start, r_total, l, pq, seed, walk_begin, ranges, variants, outs, ws,
                     stream, dev, world, flush, main_variant):
    """Each variant once (after an untimed run on a small range) on the same walk-id ranges; the
    rows are compared with the timed main variant's output."""
    import torch

    cnt = max(c for _, c in ranges)
    tmp = torch.empty((cnt, l), dtype=torch.int32, device=dev)
    sub = {}
    for vname in variants:
        vcode = n2v.VARIANTS[vname]
        ms, same, tr, shas = [], True, 0, []
        for i in range(len(pq)):
            def call(off, c):
                n2v.n2v_walk(graph.handle, starts, n_start, r_total, l, pq[i][0], pq[i][1], seed, walk_begin + off,
                             c, tmp[:c], ws, vcode, stream)

            call(ranges[0][0], min(ranges[0][1], 4096))  # warm-up: module load, function attributes
            torch.cuda.synchronize(dev)
            flush.fill_(7)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h = hashlib.sha256()
            t_ms = 0.0
            for off, c in ranges:
                a.record(stream)
                call(off, c)
                b.record(stream)
                torch.cuda.synchronize(dev)
                t_ms += a.elapsed_time(b)
                same &= bool(torch.equal(tmp[:c], outs[i][off:off + c]))
                tr += n2v.traffic(graph, starts, walk_begin + off, tmp[:c])[0]
                h.update(tmp[:c].cpu().numpy().tobytes())
            ms.append(t_ms)
            shas.append(h.hexdigest())
        sub[vname] = {"value": tr * world / (sum(ms) / 1e3), "unit": UNIT, "ms": sum(ms),
                      "bit_identical_to_timed_" + main_variant: same, "rows_sha256": shas,
                      "launches": len(pq) * len(ranges) * (l if vname != "persistent" else 1)}
    del tmp
    res = {"walks_per_pq": sum(c for _, c in ranges), "ranges": ranges, "variants": sub}
    if "plain" in sub:
        res["speedup_over_plain_same_rows"] = sub[main_variant]["value"] / sub["plain"]["value"]
    if "binned" in sub:
        res["speedup_over_binned_same_rows"] = sub[main_variant]["value"] / sub["binned"]["value"]
    return res


def c2_block(n2v, dev, stream, flush, check_oracle: bool) -> dict:
    """R-MAT scale 20 (r = 10, l = 80, three (p, q)): the persistent sampler (autotuned) beside the
    binned and plain samplers on the same rows -- the first round of walk ids, every vertex once --
    with the rows of all three compared, and sampled rows checked against the oracle."""
    import numpy as np
    import torch

    from paper_1805_00280_gb300 import graphs as G

    wl = G.WORKLOADS["rmat20"]
    g = G.workload_graph("rmat20")
    graph = n2v.Graph.from_csr(g, tune=n2v.default_tune(**WORKLOAD_DEFAULTS["rmat20"]["tune"]), device=dev)
    W = g.n  # the first round: walk ids [0, n)
    n2v.autotune(graph, np.arange(g.n, dtype=np.int32), 20, wl.pq[0][0], wl.pq[0][1], wl.seed,
                 sample=min(1 << 20, g.n), stream=stream)
    starts = torch.arange(g.n, dtype=torch.int32, device=dev)
    ws_bytes = max(n2v.n2v_walk_ws_bytes(graph.handle, W, wl.l, n2v.N2V_PERSISTENT), 256)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.int64, device=dev)
    outs = [torch.empty((W, wl.l), dtype=torch.int32, device=dev) for _ in wl.pq]
    for i, (p, q) in enumerate(wl.pq):
        n2v.n2v_walk(graph.handle, starts, g.n, wl.r, wl.l, p, q, wl.seed, 0, W, outs[i], ws, n2v.N2V_PERSISTENT,
                     stream)
    torch.cuda.synchronize(dev)
    res = compare_variants(n2v, graph, starts, g.n, wl.r, wl.l, wl.pq, wl.seed, 0, [(0, W)],
                           ["persistent", "binned", "plain"], outs, ws, stream, dev, 1, flush, "persistent")
    res.update({"workload": "rmat20", "desc": wl.note, "n": g.n, "nnz": g.nnz, "pq": wl.pq,
                "tune": graph.tune.as_dict()})
    if check_oracle:
        ok, nrows = True, 0
        rng = np.random.default_rng(20)
        hubs = np.sort(np.argsort(g.degrees(), kind="stable")[-64:])
        ids = np.unique(np.concatenate([rng.choice(W, size=2048, replace=False), hubs]))
        for i, (p, q) in enumerate(wl.pq):
            want = oracle_mod().walk(g.row_ptr, g.col, None, np.arange(g.n, dtype=np.int32), wl.l, p, q, wl.seed,
                                     ids, threads=os.cpu_count() or 1)
            ok &= bool(np.array_equal(outs[i][torch.from_numpy(ids).to(dev)].cpu().numpy(), want))
            nrows += len(ids)
        res["parity"] = {"oracle_rows_checked": nrows, "bit_exact": ok}
    del outs
    graph.close()
    return res


def stored_compare(n2v, graph, g, starts, n_start, r_total, l, pq, seed, walk_begin, Wc, outs, stream, dev, world,
                   flush):
    """The stored-table baseline (Section 3.2, Eq. 1) beside the on-the-fly sampler.

    Reports the table's bytes against the graph's, and where the table fits in
    half the free device memory, its build time and its walk rate on the same
    rows (which must be identical)."""
    import torch

    tbytes, entries = n2v.n2v_stored_bytes(graph.handle, stream)
    gbytes = 8 * (g.n + 1) + 4 * g.nnz + (12 * g.nnz if g.w is not None else 0)
    res = {"table_bytes": tbytes, "eq1_bytes": 8 * entries, "graph_bytes": gbytes,
           "table_over_graph": tbytes / gbytes}
    free, _ = torch.cuda.mem_get_info(dev)
    if tbytes > free // 2:
        res["fits"] = False
        return res
    res["fits"] = True
    tmp = torch.empty((Wc, l), dtype=torch.int32, device=dev)
    build_ms, ms, same, tr = [], [], True, 0
    for i in range(len(pq)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        table = n2v.StoredTable(graph, pq[i][0], pq[i][1], stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        build_ms.append(a.elapsed_time(b))
        launch = lambda: n2v.n2v_stored_walk(graph.handle, table.buf, starts, n_start, r_total, l, seed, walk_begin,
                                             Wc, tmp, stream)
        launch()  # warm-up
        torch.cuda.synchronize(dev)
        flush.fill_(7)
        a.record(stream)
        launch()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
        same &= bool(torch.equal(tmp, outs[i][:Wc]))
        tr += n2v.traffic(graph, starts, walk_begin, tmp)[0]
        del table
    res.update({"value": tr * world / (sum(ms) / 1e3), "unit": UNIT, "ms": sum(ms), "build_ms": build_ms,
                "bit_identical_to_timed": same})
    return res


def ingest_ncu(csv_path: str, json_path: str, out_dir: str | None = None) -> str:
    """Per-call DRAM traffic of the timed sampler launches, from a one-pass ncu launch list.

    The run must be ``bench.py ... --no-cpu --no-e2e --compare none --c2 0`` (one variant timed,
    nothing after the timed region but the traffic counters), captured with
    ``--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum``.  Its last
    steps x len(pq) x chunks sampler launches are the timed ones; one timed unit (the roofline's
    "launch") is one n2v_walk call, i.e. ``chunks`` kernel launches, and its traffic is their sum.
    """
    import csv

    line = [x for x in open(json_path) if x.startswith("{")][-1]
    d = json.loads(line)
    cfg = d["config"]
    npq, steps = len(cfg["pq"]), d["steps"]
    kernel = d["roofline"]["kernel"]
    chunk = cfg["tune"].get("chunk_walkers", 0)
    per_call = -(-cfg["walks_per_gpu"] // chunk) if chunk > 0 and cfg["variant"] == "persistent" else 1
    rows = list(csv.reader(open(csv_path)))
    hi = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    h = rows[hi]
    I, K, MN, MV = (h.index(x) for x in ("ID", "Kernel Name", "Metric Name", "Metric Value"))
    by = {}
    for r in rows[hi + 1:]:
        if len(r) > MV and kernel in r[K]:
            by.setdefault(int(r[I]), {})[r[MN]] = float(r[MV].replace(",", ""))
    launches = [by[i] for i in sorted(by)]
    timed = launches[-steps * npq * per_call:]
    calls = [timed[c * per_call:(c + 1) * per_call] for c in range(steps * npq)]
    traffic = [sum(x["dram__bytes_read.sum"] + x["dram__bytes_write.sum"] for x in c) for c in calls]
    out = {"workload": cfg["workload"], "variant": cfg["variant"], "kernel": kernel, "csrc_sha": csrc_digest(),
           "tune": cfg["tune"], "pq": cfg["pq"], "walks_per_call": cfg["walks_per_gpu"],
           "kernel_launches_per_call": per_call,
           "dram_bytes_per_launch": int(statistics.mean(traffic)),
           "per_call": [{"dram_read": int(sum(x["dram__bytes_read.sum"] for x in c)),
                         "dram_write": int(sum(x["dram__bytes_write.sum"] for x in c)),
                         "ncu_ms": sum(x["gpu__time_duration.sum"] for x in c) / 1e6} for c in calls],
           "algorithmic_bytes_per_launch": d["roofline"]["algorithmic_bytes_per_launch"],
           "source": "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                     "--clock-control none (one pass), the timed launches of bench.py --workload %s --steps %d "
                     "--warmup %d --no-cpu --no-e2e --compare none --c2 0" % (cfg["workload"], steps, d["warmup"])}
    p = os.path.join(out_dir or os.path.join(REPO, "profiles"), f"traffic_{cfg['variant']}_{cfg['workload']}.json")
    with open(p, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({"written": p, "dram_bytes_per_launch": out["dram_bytes_per_launch"]}))
    return p


def main():
    args = parse_args()
    if args.ingest_ncu:
        ingest_ncu(*args.ingest_ncu)
    elif args.sweep:
        from paper_1805_00280_gb300 import graphs as G

        if args.gpus > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            raise SystemExit("--sweep runs on one GPU")
        for name in G.SWEEPS[args.sweep]:
            args.workload = name
            run_ours(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "rmat24serve":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
