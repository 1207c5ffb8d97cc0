"""The JSON line of bench.py's reference arm, on the CPU.

`bench.py --impl reference` times the oracle on the host cores, on a bounded
sample of the benchmark's scene, and prints the same line as the library's
arm with "impl": "reference", a cpu_baseline describing the run and an e2e
block with no host-device traffic. Under torchrun only rank 0 runs it; the
other ranks exit 0 without work. Fewer than three warm-up steps are refused.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None, timeout=600):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, env=e, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_complete_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key, typ in [("metric", str), ("unit", str), ("dtype", str), ("data", str), ("scaling", str),
                     ("n_gpus", int), ("steps", int), ("warmup", int)]:
        assert isinstance(d[key], typ), key
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 3)
    assert d["data"] == "synthetic" and isinstance(d["config"]["workload"], str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and isinstance(cb["sample"], str)
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3", env={"RANK": "1", "WORLD_SIZE": "2"},
               timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("impl", ["reference", "ours"])
def test_fewer_than_three_warmup_steps_are_refused(impl):
    r = _bench("--impl", impl, "--steps", "1", "--warmup", "2", timeout=120)
    assert r.returncode == 2 and "--warmup must be at least 3" in r.stderr
