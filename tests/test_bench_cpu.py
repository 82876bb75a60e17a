"""Host-side helpers of bench.py that need no GPU.

The roofline's `traffic` comes from a committed ncu record and is reported
only while the kernel's source is unchanged since the capture; the peak
comes from the measured peaks file, with the documented fallback."""

import hashlib
import json

import pytest


def _tree(tmp_path, src_text, recorded_text):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text(src_text)
    sha = hashlib.sha256(recorded_text.encode()).hexdigest()
    rec = {"pm_x": {"bytes_per_launch": 123, "source": "k.cu", "source_sha256": sha}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))


def test_traffic_reported_while_the_source_matches(tmp_path, monkeypatch):
    import bench
    _tree(tmp_path, "kernel v1", "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("pm_x") == 123
    assert bench.recorded_traffic("pm_other") is None


def test_traffic_dropped_once_the_source_changes(tmp_path, monkeypatch):
    import bench
    _tree(tmp_path, "kernel v2", "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("pm_x") is None


def test_traffic_absent_without_a_record(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("pm_x") is None


def test_peak_from_the_measured_file_else_fallback(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, kind = bench.measured_peaks()
    assert kind == "fallback" and peak == pytest.approx(6800.0)
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6760.9}))
    peak, kind = bench.measured_peaks()
    assert kind == "measured" and peak == pytest.approx(6760.9)
