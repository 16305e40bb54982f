"""Host logic of bench.py that decides whether a measurement stands (no GPU):
the clock record taken during the timed region, the roofline peaks and the
DRAM-traffic lookup that is voided when a kernel's source changes."""
import json
import os

import pytest

import bench


def _sampler_with(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    assert not os.path.exists(s.path)          # the temporary record is removed


def test_clock_summary_flags_thermal_and_missing_samples(tmp_path):
    s = _sampler_with(tmp_path, [
        "0, 1500, 2070, 1000, 0x48, Active, Not Active, Active, Not Active",
        "0, [N/A], 2070, 1000, 0x48, Not Active, Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500.0 and out["samples"] == 2
    empty = bench.ClockSampler(0)
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                               "samples": 0}


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_traffic_is_voided_when_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"l2p": {"bytes_per_launch": 123, "source": "k.cu", "source_sha": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("l2p") == 123
    assert bench._traffic("p2m") is None
    src.write_text("kernel v2\n")
    assert bench._traffic("l2p") is None

