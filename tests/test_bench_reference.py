"""The benchmark's reference arm (the FP64 CPU oracle on the host cores) prints one JSON
line with the keys of the benchmark contract, on the same metric and workload config as
the GPU arm.  Runs on the CPU: the reference arm does no GPU work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(300)
def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "lg1",
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "2", "--cpu-procs", "2"]
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=280)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == "fwd+grad CRN-PF particle-steps/s" and d["unit"] == "particle-steps/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = d["config"]
    assert cfg["workload"].startswith("lg1:") and (cfg["N"], cfg["M"], cfg["T"], cfg["D"]) == (64, 128, 100, 3)
    # ms per step is the measured wall time of a step's sample (it fits the run); the time the
    # whole workload (N filters) would take at the measured rate is labelled as extrapolated
    ext = cfg["extrapolated_ms_per_iteration"]
    assert abs(ext - 1e3 * 64 * 128 * 100 / d["value"]) <= 1e-9 * ext
    assert 0 < d["ms_per_step"] * d["steps"] < 1e3 * 280
    # the oracle at one thread and on all (here: two) cores
    assert d["cpu_baseline"]["threads_1"]["threads"] == 1 and d["cpu_baseline"]["threads_1"]["value"] > 0
    assert d["cpu_baseline"]["threads_all"] == {"value": d["value"], "threads": 2}
