"""CPU: the benchmark's reference arm (the FP64 oracle timed on the host cores) prints one
JSON line with the contract's keys, and the bench's pure helpers (roofline class mapping,
per-rank throughput) behave as documented.  No GPU is touched."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.timeout(600)
def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is False and d["unit"] == "s"
    assert d["config"]["workload"] == "chem_L16_D256"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the timed region is the oracle work actually done, not the extrapolated value
    assert d["ms_per_step"] * d["steps"] / 1e3 <= d["timed_wall_s"] * 1.01 + 1e-3


def test_stopping_rule():
    import bench
    assert not bench.rule_met([-1.0])
    assert not bench.rule_met([-21.0, -21.1])
    assert bench.rule_met([-21.1, -21.1 - 1e-5])            # 4.7e-7 relative
    assert not bench.rule_met([-21.1, -21.1 - 3e-5])        # 1.4e-6 relative
    assert bench.rule_met([-5.0, -21.1, -21.1 + 1e-6])      # only the last two count


def test_roofline_class_mapping():
    import bench
    peaks = dict(hbm=6782.1, bf16_sus=1726.0, bf16=1918.6, src="test")
    d = dict(ms=2.0, flops=4e12, bytes=8e9, launches=1)
    assert bench.class_roofline("emu_s1", d, peaks, "bf16")[0] == "tensor"
    b, u, p, a = bench.class_roofline("emu_s3", d, peaks, "bf16")
    assert (b, u, p) == ("hbm", "GB/s", 6782.1) and abs(a - 4000.0) < 1e-9
    assert bench.class_roofline("svd", d, peaks, "bf16")[0] == "alu"
    assert "svd" in bench.LATENCY_BOUND and "lq" in bench.LATENCY_BOUND
    for k, r in bench.DRAM_TRAFFIC_RATIO.items():
        assert 0.5 < r < 5.0, k


def test_profile_modes_and_traffic_sources():
    """The profiling modes parse, and every class with a DRAM traffic ratio names the
    committed profile summary it was measured in."""
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--profile-svd", "--reps", "2"]
        a = bench.parse()
        assert a.profile_svd and a.reps == 2 and not a.profile_env
        sys.argv = ["bench.py", "--profile-env", "--D", "256"]
        a = bench.parse()
        assert a.profile_env and a.D == 256
    finally:
        sys.argv = old
    for k in bench.DRAM_TRAFFIC_RATIO:
        src = bench.DRAM_TRAFFIC_CAPTURE[k]
        assert os.path.isfile(os.path.join(ROOT, src)), src
