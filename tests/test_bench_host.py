"""Host-side parts of bench.py, on the CPU: the reference arm's JSON line,
the traffic lookup keyed by (kernel, angles, workload), and the clock
window's filtering of nvidia-smi samples (fed with recorded lines)."""
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.join(os.path.dirname(__file__), "..")
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gelem/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["metric"] == bench.METRIC


def test_traffic_lookup_is_exact_and_plausible():
    n = 1 << 28
    b, src = bench.lookup_traffic("sincos_f32", n, "bandwidth")
    assert src and 0.9 * 12 * n <= b <= 1.1 * 12 * n
    for name in ("sin_f32", "cos_f32", "tan_f32", "taylor_sin_f32"):
        b, _ = bench.lookup_traffic(name, n, "bandwidth")
        assert 0.9 * 8 * n <= b <= 1.1 * 8 * n
    assert bench.lookup_traffic("sincos_f32", n // 4, "bandwidth") == (None, None)
    assert bench.lookup_traffic("sincos_f32", n, "large") == (None, None)


class _FakeProc:
    pass


def test_clock_window_keeps_only_samples_inside_the_window():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    t = time.perf_counter()
    c.lines = [(t - 5.0, "0, 1000, 2070, 900, 0x4, Active, Not Active, Not Active, Not Active"),
               (t, "0, 2070, 2070, 1200, 0x0, Not Active, Not Active, Not Active, Active"),
               (t + 0.1, "0, 2060, 2070, 1250, 0x0, Not Active, Not Active, Not Active, Not Active"),
               (t + 0.2, "0, 2070, 2070, 1250, 0x0, Not Active, Not Active, Not Active, Not Active"),
               (t + 9.0, "0, 900, 2070, 500, 0x0, Not Active, Active, Not Active, Not Active")]
    w = c.window(t, t + 0.2)
    assert w["samples"] == 3 and w["sm_mhz"] == 2070.0 and w["sm_max_mhz"] == 2070.0
    assert w["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).window()["reasons"] == ["nvidia-smi unavailable"]
