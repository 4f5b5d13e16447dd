"""CPU checks of bench.py: the reference arm (the oracle timed on host cores)
prints one JSON line with the keys of the benchmark contract, and the
synthetic workloads are built as their recipes state (seeded, with the
stated sizes), without a GPU."""
import json
import os
import subprocess
import sys

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e")


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "qc96", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == os.cpu_count()
    assert d["cpu_baseline"]["nproc"] == os.cpu_count()
    assert d["config"]["workload"] == "qc96"


def test_serving_stream_recipe():
    codes, jobs = bench.serve_jobs(200)
    assert len(codes) == 8 and all(c.n <= 10_000 for c in codes)
    kinds = [j[0] for j in jobs]
    assert 0.6 < kinds.count("enum") / len(jobs) < 0.9
    for kind, c, p in jobs:
        assert 0 <= c < len(codes)
        if kind == "enum":
            assert 1_000 <= p["cand_end"] <= 100_000 and p["max_size"] == 2
        else:
            assert p["n_samples"] == 1_000_000 and 3.0 <= p["ebn0_db"] <= 5.0
    # seeded: the same stream twice
    assert bench.serve_jobs(200)[1] == jobs


def test_batch_workload_recipe():
    w = bench.workload_for("batch32", 0)
    assert w["code"].name == "batch100" and w["max_size"] == 2 and w["K"] == 20
    shifts = w["code"].shifts
    assert shifts.shape[0] == 4 and 16 <= shifts.shape[1] <= 32
    assert np.all(shifts < w["code"].Z)


def test_served_launch_count():
    jobs = [("enum", 0, dict(cand_end=40_000)), ("is", 1, dict(n_samples=1_000_000)),
            ("enum", 2, dict(cand_end=1_000))]
    res = [{"enum_stats": {"n_cand": 40_000}}, {"enum_stats": {"n_cand": 0}}, {"enum_stats": {"n_cand": 700}}]
    # 3 + ceil(40000/16384) + 3 = 9; ceil(10^6/32768) + 2 = 33; 3 + 1 + 3 = 7
    assert bench.served_launches(jobs, res) == 9 + 33 + 7


def test_alu_roofline_terms():
    # two values per 16-bit-pair lane operation, 12 operations and 4 shared-memory bytes per edge update
    pk = dict(num_sms=2, int32_ops_per_clk_sm=128.0, u16x2_ops_per_clk_sm=128.0, smem_bytes_per_clk_sm=128.0)
    r = bench.alu_roofline(eu_per_launch=1e9, ms_launch=100.0, pk=pk, sm_mhz=1000.0)
    clk = 2 * 1e9
    assert r["terms"]["int_bound"] == 128 * clk * 2 / 12
    assert r["terms"]["smem_bound"] == 128 * clk / 4
    assert r["peak"] == min(r["terms"]["int_bound"], r["terms"]["smem_bound"])
    assert r["achieved"] == 1e10 and abs(r["frac"] - 1e10 / r["peak"]) < 1e-12
    r1 = bench.alu_roofline(1e9, 100.0, pk, 1000.0, packed=False)
    assert r1["peak"] == 128 * clk / 12
