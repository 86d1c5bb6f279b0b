"""Host-side logic of bench.py, no GPU: picking the timed launches out of an ncu launch list."""
import csv
import json

import bench


def write_launch_list(path, kernels):
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for i, (name, ns, rd, wr) in enumerate(kernels):
            w.writerow([i, name, "gpu__time_duration.sum", "ns", f"{ns:,}"])
            w.writerow([i, name, "dram__bytes_read.sum", "byte", f"{rd:,}"])
            w.writerow([i, name, "dram__bytes_write.sum", "byte", f"{wr:,}"])


def test_ingest_picks_the_timed_launches(tmp_path):
    """One n2v_walk call per (p, q); nothing but the traffic counters after the timed steps."""
    K = "void n2v::k_persistent<5>(n2v::GraphView, ...)"
    npq, warmup, steps = 3, 3, 1
    launches = [(K, 10, 1, 1)] * 4  # autotuner
    launches += [("n2v::k_validate_stats", 5, 0, 0)]
    launches += [(K, 100 + i, 7, 1) for i in range(warmup * npq)]  # warm-up
    launches += [("at::fill", 1, 0, 0)]
    launches += [(K, 200 + i, 1000 * (i + 1), 10 * (i + 1)) for i in range(steps * npq)]  # timed
    launches += [("n2v::k_traffic", 9, 0, 0)] * npq
    write_launch_list(tmp_path / "l.csv", launches)
    line = {"steps": steps, "warmup": warmup,
            "config": {"pq": [[1, 1], [0.25, 4], [4, 0.25]], "workload": "testwl", "variant": "persistent",
                       "tune": {"blocks_per_sm": 5, "chunk_walkers": 0}, "walks_per_gpu": 64},
            "roofline": {"kernel": "k_persistent", "algorithmic_bytes_per_launch": [1, 2, 3]}}
    (tmp_path / "b.json").write_text("some log line\n" + json.dumps(line) + "\n")
    p = bench.ingest_ncu(str(tmp_path / "l.csv"), str(tmp_path / "b.json"), str(tmp_path))
    d = json.load(open(p))
    assert d["kernel_launches_per_call"] == 1
    assert [x["dram_read"] for x in d["per_call"]] == [1000, 2000, 3000]
    assert [x["dram_write"] for x in d["per_call"]] == [10, 20, 30]
    assert d["dram_bytes_per_launch"] == (1010 + 2020 + 3030) // 3
    assert d["tune"] == {"blocks_per_sm": 5, "chunk_walkers": 0} and d["csrc_sha"] == bench.csrc_digest()


def test_ingest_sums_the_chunk_launches_of_a_call(tmp_path):
    """A call of 2^26 walks in 2^23-walk chunks is eight kernel launches: its traffic is their sum."""
    K = "void n2v::k_persistent<5>(n2v::GraphView, ...)"
    launches = [(K, 10, 1, 1)] * 5  # autotuner
    launches += [(K, 100, 7, 7)] * 8  # warm-up call
    launches += [(K, 200, 100 + i, 1) for i in range(8)]  # the timed call
    launches += [("n2v::k_traffic", 9, 0, 0)]
    write_launch_list(tmp_path / "l.csv", launches)
    line = {"steps": 1, "warmup": 1,
            "config": {"pq": [[2, 0.5]], "workload": "big", "variant": "persistent",
                       "tune": {"chunk_walkers": 1 << 23}, "walks_per_gpu": 1 << 26},
            "roofline": {"kernel": "k_persistent", "algorithmic_bytes_per_launch": [1]}}
    (tmp_path / "b.json").write_text(json.dumps(line) + "\n")
    d = json.load(open(bench.ingest_ncu(str(tmp_path / "l.csv"), str(tmp_path / "b.json"), str(tmp_path))))
    assert d["kernel_launches_per_call"] == 8
    assert d["dram_bytes_per_launch"] == sum(100 + i for i in range(8)) + 8


def test_traffic_tuning_compares_effective_tunings():
    """A capture at the default 20 warps per SM (blocks_per_sm 0) matches a run whose tuner chose 5."""
    a = {"blocks_per_sm": 0, "stream_ratio": 100}
    assert bench.effective_tune(a) == bench.effective_tune({"blocks_per_sm": 5, "stream_ratio": 100})
    assert bench.effective_tune(a) != bench.effective_tune({"blocks_per_sm": 4, "stream_ratio": 100})
    assert bench.effective_tune(None) is None


def test_ingest_takes_every_instance_of_the_kernel(tmp_path):
    """The lean instances' names carry a second template argument (with a comma)."""
    K = "void n2v::k_persistent<5, 2>(n2v::GraphView, n2v::WalkJob, unsigned long long *, n2v::LaunchCfg, unsigned int *)"
    launches = [(K, 100, 7, 7)] * 2  # warm-up call
    launches += [(K, 200, 50 + i, 2) for i in range(2)]  # the timed call
    write_launch_list(tmp_path / "l.csv", launches)
    line = {"steps": 1, "warmup": 1,
            "config": {"pq": [[2, 0.5]], "workload": "w", "variant": "persistent",
                       "tune": {"chunk_walkers": 4}, "walks_per_gpu": 8},
            "roofline": {"kernel": "k_persistent", "algorithmic_bytes_per_launch": [1]}}
    (tmp_path / "b.json").write_text(json.dumps(line) + "\n")
    d = json.load(open(bench.ingest_ncu(str(tmp_path / "l.csv"), str(tmp_path / "b.json"), str(tmp_path))))
    assert d["kernel_launches_per_call"] == 2
    assert d["dram_bytes_per_launch"] == 50 + 51 + 2 * 2


def test_dram_fraction():
    """The R-MAT 26 capture: 144.91 TB a call over 35.873 s is 59% of 6,798.9 GB/s."""
    d = bench.dram_fraction(144_910_358_544_640, [35_872.9], 6798.9)
    assert abs(d["achieved"] - 4039.6) < 1.0 and abs(d["frac"] - 0.594) < 0.001
    assert bench.dram_fraction(None, [1.0], 6798.9) is None
    assert bench.dram_fraction(10, [], 6798.9) is None
    two = bench.dram_fraction(2e9, [1.0, 3.0], 1000.0)  # per-call bytes, mean over two calls
    assert abs(two["achieved"] - 1000.0) < 1e-9  # 4 GB in 4 ms
