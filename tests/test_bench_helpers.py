"""Host-side helpers of bench.py: the roofline object of each kernel class
(bound, unit, peak and the fraction achieved/peak) and the peaks it reads."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


@pytest.mark.parametrize("name,bound,unit", [
    ("solve_gemm", "tensor", "TFLOP/s"), ("sweep_gemm", "tensor", "TFLOP/s"), ("sweep_narrow", "tensor", "TFLOP/s"),
    ("fp64_residual", "alu", "TFLOP/s"), ("fp64_path", "alu", "TFLOP/s"), ("ff_residual", "alu", "T fp32 instr/s"),
    ("panel_inverse", "alu", "TFLOP/s"), ("panel_product", "alu", "TFLOP/s"), ("schur", "alu", "TFLOP/s"),
    ("solve_coupling", "hbm", "GB/s")])
def test_roofline_classes(name, bound, unit):
    roof = bench.roofline(name, 10.0, 2.0e12, 100, PK, "fallback")
    assert roof["bound"] == bound and roof["unit"] == unit
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    if bound == "tensor":
        # split-pair products: three bf16 MMAs per product at the sustained bf16 rate
        assert roof["peak"] == pytest.approx(1700.0 / 3)
        assert roof["achieved"] == pytest.approx(2.0e12 / 10e-3 / 1e12)
        assert roof["flops_per_launch"] == pytest.approx(2.0e10)
    if bound == "hbm":
        assert roof["peak"] == 6800.0
        assert roof["achieved"] == pytest.approx(2.0e12 / 10e-3 / 1e9)
        assert roof["bytes_per_launch"] == pytest.approx(2.0e10)
    if name in ("fp64_residual", "fp64_path"):
        assert roof["peak"] == bench.FP64_PEAK_TFLOPS


def test_traffic_only_for_captured_kernels():
    for name in bench.TRAFFIC:
        roof = bench.roofline(name, 1.0, 1.0e9, 1, PK, "fallback")
        assert roof["traffic"] == bench.TRAFFIC[name] > 0
    assert bench.roofline("panel_inverse", 1.0, 1.0e9, 1, PK, "fallback")["traffic"] is None


def test_peaks_prefer_the_measured_file():
    pk, src = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and pk["hbm_gbs"] > 0 and pk["bf16_tflops_sustained"] > 0
    else:
        assert src == "fallback" and pk == bench.FALLBACK_PEAKS
