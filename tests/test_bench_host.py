"""Host-side helpers of bench.py (no GPU): the DRAM-traffic record is reported
only while the sources it was measured on are unchanged, and the roofline
peaks come from the measured file."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    rec = {"kind_a": {"bytes_per_launch": 123.0,
                      "sources": {"k.cuh": hashlib.sha256(src.read_bytes()).hexdigest()}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("kind_a") == 123.0
    assert bench.measured_traffic("kind_b") is None
    src.write_text("kernel v2\n")
    assert bench.measured_traffic("kind_a") is None


def test_peaks_are_the_measured_ones():
    pk, src = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured"
    assert pk["hbm_gbs"] > 0 and pk["bf16_tflops_sustained"] > 0
