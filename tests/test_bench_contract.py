"""The reference arm of bench.py runs on the CPU and prints the contract's JSON line."""

from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["batch64", "poisson750"])
def test_reference_arm_line(workload):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          workload, "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
    if workload == "batch64":  # the repo arm prints the same metric and workload
        sys.path.insert(0, ROOT)
        import bench
        assert line["metric"] == bench.METRIC
        assert line["config"]["workload"] == bench.recipes_for("batch64")[1]
        assert "each step" in line["config"]["sample"] and line["cpu_baseline"]["cpu_model"]


def test_cpu_sample_one_frame_per_size_class():
    sys.path.insert(0, ROOT)
    import bench
    recipes, _ = bench.recipes_for("batch64")
    sample = bench.cpu_sample(recipes)
    assert [(r["w"], r["h"]) for r in sample] == [(800, 800)] * 4
    firsts = [recipes[i] for i in (0, 16, 32, 48)]
    assert [(r["gain"], r["readnoise"], r["sky"]) for r in sample] == [(r["gain"], r["readnoise"], r["sky"])
                                                                         for r in firsts]
    # densities kept: the 4096x4096 class has 16384/625 times the 800x800 area
    assert abs(sample[3]["ncr"] - firsts[3]["ncr"] * 640000 / 4096 ** 2) <= 1
