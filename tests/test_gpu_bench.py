"""bench.py's main leg runs and prints one JSON line with the keys its contract needs (small
lattice, few steps; the full default run is the benchmark itself)."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()


@pytest.mark.parametrize("extra", [[], ["--storage", "2"], ["--step-kernel", "1"]])
def test_bench_main_leg_prints_its_line(built, extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--config", "jet96", "--only-main", "--steps", "5",
           "--warmup", "3"] + extra
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "config", "roofline", "kernels", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 5 and line["warmup"] == 3
    assert line["gpu_launches"] >= 5
    rf = line["roofline"]
    assert rf["bound"] == "hbm" and 0 < rf["frac"] < 2 and rf["peak"] > 0
