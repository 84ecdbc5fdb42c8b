"""The roofline object of the benchmark line names the kernel that runs for each precision
and divides algorithmic flops by that kernel's own peak.  Host arithmetic only."""

import numpy as np
import pytest

import bench

PEAKS = {"bf16_tflops": 2000.0}
SIZES = np.array([128.0, 300.0, 1000.0])


def test_algorithmic_flops_are_the_upper_triangle_of_each_square():
    # s (s + 1) / 2 dot products of length s, 2 s flops each, summed over the parts
    want = sum(s * (s + 1) / 2 * 2 * s for s in SIZES)
    assert bench.alg_flops(SIZES) == pytest.approx(want)
    assert bench.alg_flops(SIZES, 3) == pytest.approx(3 * want)


def test_executed_flops_cover_whole_upper_tiles():
    # one 128-part: one tile, K = 128; padding and whole diagonal tiles make it exceed s^2 (s + 1)
    assert bench.tc_exec_flops(np.array([128.0]), 64, 1) == 2 * 128 * 128 * 128
    s = np.array([300.0])
    nt = 3
    assert bench.tc_exec_flops(s, 64, 1) == nt * (nt + 1) / 2 * 2 * 128 * 128 * 320
    # trimmed: the last column block's MMAs cover 300 - 256 = 44 -> 48 columns
    assert bench.tc_exec_flops(s, 64, 1, trim=True) == (nt * (nt + 1) / 2 * 128 - nt * (128 - 48)) * 2 * 128 * 320


@pytest.mark.parametrize("prec,bound,kernel,peak", [
    ("fp64", "alu", "square_simt_kernel<double>", 2000.0 * 1.25 / 2250.0),
    ("fp64e", "tensor", "oz_step_kernel", 2000.0),
    ("fp32", "alu", "square_simt_kernel<float>", 128 * 152 * 2 * 2.07 / 1e3),
    ("tf32x3", "tensor", "square_tc_persistent_kernel<tf32,3>", 2000.0 * 1100.0 / 2250.0),
    ("fp16x3", "tensor", "square_tc_persistent_kernel<fp16,3>", 2000.0),
    ("bf16", "tensor", "square_tc_persistent_kernel<bf16,1>", 2000.0),
])
def test_step_roofline_uses_the_kernel_and_peak_of_the_precision(prec, bound, kernel, peak):
    r = bench.step_roofline(prec, SIZES, 0.5, PEAKS, "measured", "tb30k")
    assert r["bound"] == bound and r["kernel"].startswith(kernel)
    assert r["peak"] == pytest.approx(peak)
    nprod = {"fp64e": bench.OZ_PRODUCTS, "tf32x3": 3, "fp16x3": 3}.get(prec, 1)
    want = bench.alg_flops(SIZES, nprod) / 0.5e-3 / 1e12
    assert r["achieved"] == pytest.approx(want)
    assert r["frac"] == pytest.approx(want / peak)
    if bound == "tensor":
        assert r["executed_frac"] >= r["frac"]  # padding only adds executed work
