"""The benchmark's compositing roofline (host arithmetic, no GPU): the
reported bound is the largest of the HBM, MUFU and FP32 lower bounds, its
fraction is that bound's time over the stage's time, and the peak falls back
to the earlier copy measurement when the measured-peaks file is missing."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_hbm_binds_on_the_4k_frame():
    # a 4K frame's counts: 92.6 M keys, 11.1 M rays, 2.58 G / 0.34 G pairs
    r = bench.compositing_roofline(2.71, 92.6e6, 11.1e6, 2.58e9, 0.34e9, 6782.8, "measured")
    b = r["bounds_ms"]
    assert r["bound"] == "hbm" and b["hbm"] > b["mufu"] > b["alu"]
    # bytes: 40 B a key (8 B key, 32 B record) + 12 B a ray; the bound time
    # over the stage time
    assert abs(r["bytes_per_launch"] - (92.6e6 * 40 + 11.1e6 * 12)) < 1.0
    assert abs(r["frac"] - b["hbm"] / 2.71) < 1e-12
    assert abs(r["achieved"] - r["bytes_per_launch"] / 2.71e-3 / 1e9) < 1e-6
    assert r["unit"] == "GB/s" and r["peak"] == 6782.8
    # the FP32 view rides along: 13 ops per evaluated, 9 per composited pair
    flops = 13 * 2.58e9 + 9 * 0.34e9
    assert abs(r["alu"]["flop_per_launch"] - flops) < 1.0
    assert abs(r["alu"]["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9


def test_arithmetic_binds_when_few_bytes_move():
    # many evaluated pairs per key: MUFU binds, reported as "alu"
    r = bench.compositing_roofline(1.0, 1e6, 1e5, 5e9, 1e8, 6782.8, "measured")
    assert r["bounds_ms"]["mufu"] > r["bounds_ms"]["hbm"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["frac"] - r["bounds_ms"]["mufu"] / 1.0) < 1e-12


def test_peak_falls_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    gbs, src = bench.measured_hbm_gbs()
    assert gbs == bench.HBM_FALLBACK_GBS and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 7000.5}')
    gbs, src = bench.measured_hbm_gbs()
    assert gbs == 7000.5 and src.startswith("measured")
