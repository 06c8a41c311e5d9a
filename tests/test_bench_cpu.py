"""The benchmark's reference arm (the CPU oracle, timed on host cores) runs
and prints one JSON line of the contract on a small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_small():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "latlon_64x32x16", "--steps", "7", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = [l for l in r.stdout.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["value"] > 0
    assert d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # a step is one refinement step of the oracle's solve; value sums them
    m = d["config"]["refinement_steps"]
    assert d["steps"] == 7 and d["config"]["oracle_status"] == 0 and m >= 2
    assert d["config"]["final_rel_res"] <= 1e-10
    assert d["value"] == sum(d["config"]["step_ms_by_refinement_step"])
    assert d["ms_per_step"] * d["steps"] <= d["value"] * (d["steps"] // m + 1)
