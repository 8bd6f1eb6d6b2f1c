"""The bench's reference arm (the CPU oracle as it stands), run as the
driver runs it, on the small 3x4 workload: one JSON line with the keys the
contract asks for."""

import json
import os
import subprocess
import sys


def test_reference_arm_prints_one_contract_line(root):
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "grid3x4_m8",
           "--steps", "2", "--warmup", "1", "--ref-budget", "2"]
    out = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "grid3x4_m8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
