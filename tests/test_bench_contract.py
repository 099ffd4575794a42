"""The benchmark's reference arm and its JSON line, on the CPU.

`bench.py --impl reference` times the FP64 oracle on the host cores; it
needs no GPU, so its whole line is checked here on a small workload: one
JSON object with the keys the harness reads, the same metric and config
naming as the GPU arm, and a rate that matches its own time. The rank rule
(rank 0 prints, other ranks exit without work) is checked too.
"""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

import bench

ROOT = Path(__file__).resolve().parents[1]
ARGS = ["--impl", "reference", "--K", "4", "--T", "4096", "--n-prop", "8", "--steps", "2", "--warmup", "1"]


def _run(env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), *ARGS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_prints_one_valid_line():
    lines = [l for l in _run().splitlines() if l.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    cores = d["cpu_baseline"]["cores"]
    assert cores >= 1 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    # rate = proposals evaluated per step / mean step time
    assert abs(d["value"] - cores / (d["ms_per_step"] / 1e3)) <= 1e-9 * d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same workload naming as the GPU arm
    class A:
        K, T, n_prop = 4, 4096, 8
    assert d["config"] == bench.workload_config(A)


def test_reference_arm_other_ranks_do_no_work():
    assert _run({"RANK": "1"}).strip() == ""


def test_roofline_peaks():
    pk = ({"bf16_tflops_sustained": 1731.7, "bf16_tflops": 1932.2, "sm_max_mhz": 2070.0}, "measured")
    bound, peak, _ = bench.roofline_peak("tf32", pk)
    assert bound == "tensor" and abs(peak - 1731.7 * 1.1 / 2.25) < 1e-9
    bound, peak, _ = bench.roofline_peak("bf16", pk)
    assert bound == "tensor" and peak == 1731.7
    bound, peak, _ = bench.roofline_peak("fp32", pk)
    assert bound == "alu" and abs(peak - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
