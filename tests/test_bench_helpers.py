"""Host helpers of bench.py (no GPU): the clock record taken during the
timed region, the peak the roofline divides by, and the algorithmic bytes
of one operator apply."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, cap]


def test_clock_record_takes_the_median_and_the_reasons_seen():
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.rows = [_row(2070, 2070), _row(2040, 2070, cap="Active"), _row(2070, 2070), ["garbage"],
               ["0", "N/A", "2070", "", "", "", "", "", ""]]
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_names_every_slowdown():
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.rows = [_row(1500, 2070, hw="Active", hwt="Active", swt="Active")]
    assert cs.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_peak_is_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6756.8, "bf16_tflops": 1982.4}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6756.8, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "absent"))
    assert bench.load_peaks() == (6800.0, "fallback")


def test_fp32_peak_and_operator_bytes():
    # the nominal fallback follows the SM count and clock it is given
    assert bench.fp32_alu_peak_tflops() == pytest.approx(80.5, abs=0.05)
    assert bench.fp32_alu_peak_tflops(76, 2070.0) == pytest.approx(40.3, abs=0.05)
    # 256^2 grid, 32 sources: u, u0 in and y out (8 B each), chi (8 B) and the
    # (257 x 257) quarter spectrum (8 B) once per batch
    n = 256 * 256
    assert bench.op_bytes_c64(n, 32) == 24.0 * n * 32 + 8.0 * n + 8.0 * 257 * 257
