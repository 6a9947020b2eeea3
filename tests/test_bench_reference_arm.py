"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on the CPU:
one JSON line with the keys the measurement contract names, the native arm's
workload name and a force recipe; with the noise redrawn every step it says so."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cells", "64", *extra], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("regen", [0, 1])
def test_reference_arm_line(regen):
    import bench
    j = _run("--force-noise-regen", str(regen))
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == "RBC-steps/s"
    assert j["value"] > 0 and j["steps"] == 2 and j["warmup"] == 1 and j["higher_is_better"] is True
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["cpu_baseline"]["cores"] >= 1
    assert j["e2e"] == {"value": j["value"], "unit": "RBC-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = j["config"]
    assert cfg["workload"] == bench.workload_name(64, regen)
    assert cfg["forces"] == (bench.FORCES_REGEN if regen else bench.FORCES_FIXED)
    assert ("noise redrawn every step" in cfg["workload"]) == bool(regen)
