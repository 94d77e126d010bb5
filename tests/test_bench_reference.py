"""bench.py's reference arm (the CPU oracle) runs without a GPU and prints the
contract's JSON line, for a single instance and for the batch workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-budget", "0.5", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", ["c1", "c4"])
def test_reference_line(workload):
    d = run_reference("--workload", workload)
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["max_iters"] == 128
    if workload == "c1":  # small enough for the one complete oracle solve
        whole = d["cpu_baseline"]["whole_solve"]
        assert whole["ms"] > 0 and whole["status"] == 0 and whole["certified"] == 2
