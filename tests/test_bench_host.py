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


def test_roofline_entries_from_a_profile():
    """The roofline arithmetic of the bench line: achieved = algorithmic work
    per launch / average launch duration, frac against the stated peak, share
    = average duration x launches per step / step time."""
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    T, n = 12000, 5440
    # the split FP64 gradient product streams 7 BF16 digit planes: 14 T n bytes
    d = {"launches": 10, "total_ms": 2.0, "bytes_per_launch": 0.0}
    e = bench.roofline_entry("oz_gemm_bwd", d, pk, "measured", T, n, 100.0, 10)
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert abs(e["achieved"] - 14.0 * T * n / 200e-6 / 1e9) <= 0.1
    assert abs(e["fp64_equivalent_gbs"] - 8.0 * T * n / 200e-6 / 1e9) <= 0.1
    assert abs(e["frac"] - e["achieved"] / 6000.0) <= 1e-4
    assert abs(e["share_of_step"] - 0.02) <= 1e-9  # 0.2 ms x 10 launches / 100 ms
    # a tensor-core product: the profiler's work figure is its FLOPs, against sustained BF16
    d = {"launches": 4, "total_ms": 0.4, "bytes_per_launch": 2.0 * T * n * 576}
    e = bench.roofline_entry("gemm_tc_bf16_n192", d, pk, "measured", T, n, 100.0, 4)
    assert e["bound"] == "tensor" and e["unit"] == "TFLOP/s" and e["peak"] == 1700.0
    assert abs(e["achieved"] - 2.0 * T * n * 576 / 100e-6 / 1e12) <= 0.01
    # the N = 64 product reads its BF16 operand once: FLOPs / 64 bytes
    d = {"launches": 2, "total_ms": 0.04, "bytes_per_launch": 2.0 * T * n * 64}
    e = bench.roofline_entry("gemm_tc_bf16_n64", d, pk, "measured", T, n, 100.0, None)
    assert e["bound"] == "hbm" and e["share_of_step"] is None
    assert abs(e["achieved"] - 2.0 * T * n / 20e-6 / 1e9) <= 0.1
