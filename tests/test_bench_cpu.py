"""The bench's reference arm (the oracle on the host cores) with the third
TDI channel: one JSON line naming the channels, on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_three_channels():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--channels", "AET", "--steps",
           "1", "--warmup", "0", "--cpu-sample", "4"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert "TDI A,E,T" in d["config"]["workload"]
    assert d["cpu_baseline"]["cores"] == 2      # the threads the oracle used
