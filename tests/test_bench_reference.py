"""bench.py's reference arm on CPU: the oracle timed on the host cores, one JSON line with
the arm's metric, unit and contract keys; under a multi-rank launch only rank 0 works and
prints, the other ranks exit 0 at once."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "ssao16_256", "--steps", "2",
           "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    import bench
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == "Mpix/s"
    assert j["value"] > 0 and j["higher_is_better"] is True and j["warmup"] >= 3
    assert j["config"]["workload"] == "ssao16_256"
    # the same config dict the GPU arm prints for this workload
    import scenegen as sg
    assert j["config"] == bench.config_of("ssao16_256", dict(sg.WORKLOADS["ssao16_256"]), 0, 1)
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
