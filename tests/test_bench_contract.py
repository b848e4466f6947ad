"""The bench's reference arm (the FP64 oracle on the host cores) prints one
JSON line that keeps the benchmark contract: metric, unit and direction of
the GPU arm, a positive value, the CPU baseline it measured and an end-to-end
entry without copies. Runs on the 2-line swath with a few nodes per step."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, env=None):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return lines


def test_reference_arm_prints_one_contract_line():
    lines = _run("--impl", "reference", "--small", "--steps", "2", "--warmup", "1",
                 "--ref-nodes", "64")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "grid nodes/s (IDW k=16, kriging k=32)"
    assert d["unit"] == "nodes/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("survey swath, 2 lines")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "random nodes" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert _run("--impl", "reference", "--small", "--steps", "1", "--warmup", "0",
                "--ref-nodes", "16", env=env) == []
