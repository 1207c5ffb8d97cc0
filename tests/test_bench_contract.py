"""The JSON line of bench.py's reference arm, on the CPU.

`bench.py --impl reference` times the oracle on the host cores, on a bounded
sample of the benchmark's scene, and prints the same line as the library's
arm with "impl": "reference", a cpu_baseline describing the run and an e2e
block with no host-device traffic. Under torchrun only rank 0 runs it; the
other ranks exit 0 without work. Fewer than three warm-up steps are refused.
The host arithmetic behind the library arm's line is pinned on hand-computed
cases: the pair pass's roofline (flops per launch over the average launch
time, against the measured peak) and the summary of the clock samples taken
during the timed region (median clock, throttle reasons seen).
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


def test_pair_roofline_arithmetic():
    """Two launches of 10 ms over 2e8 listed pairs: 1e8 pairs per launch.
    FP64: 110 flops a pair, 1.1e10 flops in 10 ms = 1.1 TFLOP/s, against the
    measured 1.186. Mixed: 155.5 flops, 1.555 TFLOP/s against 72.4. Double
    float: 682 FP32 instructions, 6.82 Top/s against 36.2. The pair pass's
    share is its 20 ms of the 30 ms profiled."""
    sys.path.insert(0, ROOT)
    import bench
    m = {"prof": {"pair": (20.0, 2), "nlist": (6.0, 2), "other": (4.0, 7)},
         "sp0": {"pairs": 5}, "sp1": {"pairs": 5 + 2 * 10**8}}
    for prec, achieved, peak in [("fp64", 1.1, 1.186), ("mixed", 1.555, 72.4), ("df64", 6.82, 36.2)]:
        r = bench.pair_roofline(m, 3, 0, prec, "dam3d")
        assert r["pairs_per_launch"] == 10**8 and r["avg_launch_ms"] == 10.0
        assert r["achieved"] == pytest.approx(achieved, rel=1e-4)
        assert r["peak"] == pytest.approx(peak)
        assert r["frac"] == pytest.approx(achieved / peak, abs=1e-4)
        assert r["share_of_step"] == pytest.approx(2 / 3, abs=1e-4)
        assert r["bound"] == "alu"


def test_clock_samples_are_summarised_with_their_throttle_reasons(tmp_path):
    """nvidia-smi rows (SM MHz, max MHz, power, reasons word, then the four
    reasons): the median SM clock, the first row's maximum, the largest
    power reading, and every reason seen active in any row. Rows that do not
    start with a number (a header, an error line) are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    rows = ["clocks.current.sm [MHz], clocks.max.sm [MHz], ...",
            "2070, 2070, 510.25, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "1980, 2070, 1398.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "2055, 2070, [N/A], 0x0000000000000008, Active, Not Active, Not Active, Not Active",
            "Unable to determine the device handle"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    s = cs.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["power_w_max"] == pytest.approx(1398.5)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not p.exists()
    empty = bench.ClockSampler(0)
    q = tmp_path / "none.csv"
    q.write_text("")
    empty.path = str(q)
    assert empty.summary()["reasons"] == ["no samples"]


def test_algorithmic_bytes_and_error_measure():
    """HBM bytes per fluid particle-step, per stage: keys (8d + 4), three
    16-byte sort passes (48), the reorder read and write (2 (24d + 18)), the
    pair pass's reads and writes (16 (2d + 2)) and the update (16 (2d + 1));
    two stages: 3D 2 x 496 = 992, 2D 2 x 376 = 752. The bench's error measure
    is the tests' max |a - b| / max(max |b|, scale), and an empty field has
    no error."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from tests.helpers import scaled_err
    assert bench.algorithmic_bytes_per_particle_step(3) == 992
    assert bench.algorithmic_bytes_per_particle_step(2) == 752
    rng = np.random.default_rng(3)
    for scale in (1e-3, 1.0, 1e3):
        a, b = rng.normal(size=(3, 50)), rng.normal(size=(3, 50))
        assert bench.scaled_err(a, b, scale) == scaled_err(a, b, scale)
    assert bench.scaled_err(np.zeros(0), np.zeros(0), 1.0) == 0.0
    assert bench.scaled_err([1.0, 2.0], [1.0, 4.0], 1.0) == 0.5
    assert bench.scaled_err([1.0, 2.0], [1.0, 2.5], 10.0) == 0.05
