"""Host-side arithmetic of the benchmark's roofline entries, on CPU.

`bench.kernel_rooflines` turns per-stage event times and the engine's work
figures into achieved rates, fractions of the measured peaks and DRAM
traffic per launch; these checks pin that arithmetic with made-up inputs.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2000.0}
WORK = {"pairs": 5e9, "sort_bytes": 1.2e10, "dense_flops": 2.4e13, "dense_issued": 2.6e13,
        "dense_bytes": 9e9, "rle_bytes": 6e9, "pack_bytes": 3e7, "combine_bytes": 6e8}
TIMINGS = {"pack": (0.02, 1), "dense_scatter": (3.0, 1), "dense_gemm": (8.0, 1), "sort_pass": (5.0, 18),
           "run_length": (4.0, 8), "accumulate": (10.0, 1), "diag": (0.01, 1), "combine": (0.49, 1),
           "dense_fix": (0.01, 1)}


def test_rates_and_fractions():
    r = bench.kernel_rooflines(TIMINGS, WORK, PEAKS, 152, smem_atomic_peak=1e13)
    acc = r["accumulate"]
    assert acc["achieved"] == pytest.approx(5e9 / 0.010 / 1e12)
    assert acc["peak"] == pytest.approx(10.0) and acc["frac"] == pytest.approx(0.05)
    assert acc["peak_source"].startswith("measured")
    gemm = r["dense_gemm"]
    assert gemm["achieved"] == pytest.approx(2.4e13 / 0.008 / 1e12)
    assert gemm["peak"] == pytest.approx(3800.0)
    sort = r["sort_pass"]
    assert sort["achieved"] == pytest.approx(1.2e10 / 0.005 / 1e9)
    assert sort["launch_ms"] == pytest.approx(5.0 / 18) and sort["launches"] == 18
    assert sort["frac"] == pytest.approx(sort["achieved"] / 6800.0)


def test_diag_and_combine_form_one_stage():
    r = bench.kernel_rooflines(TIMINGS, WORK, PEAKS, 152)
    assert "diag+combine" in r and "diag" not in r and "combine" not in r
    assert r["diag+combine"]["achieved"] == pytest.approx(6e8 / 0.0005 / 1e9)
    # Without a measured atomic rate the peak is the derived one.
    assert r["accumulate"]["peak"] == pytest.approx(32 * 152 * 2000e6 / 1e12)


def test_traffic_scales_with_the_units_of_the_launch():
    r = bench.kernel_rooflines(TIMINGS, WORK, PEAKS, 152, smem_atomic_peak=1e13)
    per, _ = bench.NCU_BYTES_PER_UNIT["sort_pass"]
    assert r["sort_pass"]["traffic"] == pytest.approx(per * 1.2e10 / 18)
    per, _ = bench.NCU_BYTES_PER_UNIT["accumulate"]
    assert r["accumulate"]["traffic"] == pytest.approx(per * 5e9)
    assert r["pack"]["traffic"] is None
    for name in ("sort_pass", "run_length", "accumulate", "dense_gemm", "dense_scatter"):
        assert r[name]["traffic_source"].startswith("profiles/")
