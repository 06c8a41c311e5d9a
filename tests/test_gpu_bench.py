"""The benchmark's GPU arm prints one JSON line of the contract (metric,
value, timing keys, roofline with live kernel timing against the measured
peak, cpu_baseline from the oracle, end-to-end timing with host buffers,
launch count, clock samples) on a small workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_gpu_arm_small():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload",
                        "latlon_256x128x32", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["unit"] == "ms" and d["higher_is_better"] is False and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "latlon_256x128x32"
    assert d["config"]["mixed_rel_res"] <= 1e-10 and d["config"]["fp64_rel_res"] <= 1e-10
    rl = d["roofline"]
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and rl["achieved"] > 0
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-9
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 256 * 128 * 32 * 8
    assert d["gpu_launches"] > 0
    assert d["clocks"]["sm_max_mhz"] > 0
