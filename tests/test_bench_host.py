"""Host logic of bench.py that needs no GPU: traffic scaling, the whole-job aggregate and the
reference arm (the FP64 oracle on the host cores), whose JSON line the contract fixes."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_scaling_per_direction():
    # forward: the volume is re-read once per 16-view chunk, projections written per view
    c = bench.NCU["exact project"]
    assert bench.full_launch_traffic("exact project", 496) == pytest.approx(
        c["dram_read_8"] * 31 + c["dram_write_8"] * 62)
    # adjoint: the projection tiles are read per view, the volume written once
    c = bench.NCU["relaxed backproject"]
    assert bench.full_launch_traffic("relaxed backproject", 496) == pytest.approx(
        c["dram_read_8"] * 62 + c["dram_write_8"])


def test_aggregate_counts_every_replica():
    assert bench.aggregate_gvv_s(2e9, 3, 1500.0, 4) == pytest.approx(4 * 2e9 * 3 / 1.5 / 1e9)


def test_counts_are_consistent():
    for name, c in bench.NCU.items():
        assert c["flop_per_vv"] > 0 and c["warp_per_vv"] > 0 and 0 < c["simt"] <= 1, name


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [line for line in out.stdout.splitlines() if line.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"] == bench.bench_config(bench.default_args(), 1)
