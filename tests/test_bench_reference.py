"""The oracle arm of bench.py (`--impl reference`) on the host: one JSON line
with the same metric, unit and direction as the GPU arm, the oracle described
as the CPU baseline, and an end-to-end figure with no device copies; under a
multi-rank launch only rank 0 works and prints."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD
    # the config names the workload only, so both arms print the same object
    assert set(d["config"]) == {"workload", "gaussians", "width", "height", "l2", "parallelism"}
    assert d["config"]["gaussians"] == 1_200_000 and d["config"]["width"] == d["config"]["height"] == 1024
    # the step time is the measured wall time of a full-frame step, not an extrapolation
    lo, hi = d["wall_s_min_max"]
    assert lo * 1e3 - 1 <= d["ms_per_step"] <= hi * 1e3 + 1      # the range is rounded to 0.1 ms
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
