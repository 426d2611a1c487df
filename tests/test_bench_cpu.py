"""Host-side arithmetic of bench.py: the roofline of the dominant kernel, the
step roofline model, the oracle's linear extrapolation in M and the lookup
of the measured traffic (tied to the tensor-core source it was taken on)."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from synth import workloads as wl  # noqa: E402

W = wl.WORKLOADS["planted-n16384-m1m-r256"]
# the machine's measured peaks: at r = 256 (256 flop per byte of O) the sustained tensor rate
# puts the ridge at 1728 / 6.68 = 259 flop/B, so the O passes are (just) bandwidth-bound
PEAKS = {"hbm_gbs": 6682.5, "bf16_tflops": 1877.8, "bf16_tflops_sustained": 1728.0}


def args(**kw):
    a = argparse.Namespace(dtype="bf16", path="step", rssr_q=2, m=None)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_roofline_is_algorithmic_bytes_over_launch_time():
    # pass A: 3 launches in 18.0 ms -> 6 ms each; bytes of O = N M 2
    prof = {"pass_A": (18.0, 3), "pass_B": (12.0, 2)}
    r = bench.roofline_for(W, args(), prof, 1, PEAKS, "tcgen05")
    assert r["kernel"] == "pass_A" and r["bound"] == "hbm"
    assert r["algorithmic_per_launch"] == W.N * W.M * 2
    assert r["achieved"] == pytest.approx(W.N * W.M * 2 / 6e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6682.5)
    # the dominant kernel is the one with the larger total time
    r = bench.roofline_for(W, args(), {"pass_A": (10.0, 2), "pass_B": (12.0, 2)}, 1, PEAKS, "tcgen05")
    assert r["kernel"] == "pass_B" and r["ms_per_launch"] == pytest.approx(6.0)
    # the FP32 SIMT engine is bound by FFMA throughput
    r = bench.roofline_for(W, args(dtype="f32"), prof, 1, PEAKS, "simt")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2.0 * W.N * W.M * W.r / 6e-3 / 1e12)


def test_roofline_above_the_ridge_is_the_tensor_rate():
    # r = 512: 512 flop per byte of O, above the ridge: tensor-bound
    w512 = wl.WORKLOADS["planted-n16384-m1m-r512"]
    prof = {"pass_A": (39.0, 3), "pass_B": (24.0, 2)}
    r = bench.roofline_for(w512, args(), prof, 1, PEAKS, "tcgen05")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == 1728.0
    assert r["achieved"] == pytest.approx(2.0 * w512.N * w512.M * w512.r / 13e-3 / 1e12)
    assert r["frac_rated"] == pytest.approx(r["achieved"] / 2250.0)


def test_step_roofline_counts_the_o_passes():
    t_bytes = W.N * W.M * 2 / (6682.5e9)
    t_flop = 2.0 * W.N * W.M * W.r / 1728.0e12
    assert bench.step_roofline_ms(W, args(), PEAKS) == pytest.approx(5 * max(t_bytes, t_flop) * 1e3)
    assert bench.step_roofline_ms(W, args(path="rssr", rssr_q=0), PEAKS) == pytest.approx(
        2 * max(t_bytes, t_flop) * 1e3)


def test_linear_fit_extrapolates_through_both_points():
    assert bench.linear_fit(2.0, 512, 5.0, 2048, 512) == pytest.approx(2.0)
    assert bench.linear_fit(2.0, 512, 5.0, 2048, 2048) == pytest.approx(5.0)
    assert bench.linear_fit(2.0, 512, 5.0, 2048, 3584) == pytest.approx(8.0)
    # a noisy negative slope is clamped: never extrapolate below the measured step
    assert bench.linear_fit(5.0, 512, 4.0, 2048, 10 ** 6) == pytest.approx(5.0)


def test_measured_traffic_is_tied_to_the_kernel_source():
    t = bench.measured_traffic(W, "pass_A")
    if t is not None:  # committed capture matches the current source
        assert t > W.N * W.M * 2  # at least the bytes of O
    small = wl.small_planted(1000, 2048, 32)
    assert bench.measured_traffic(small, "pass_A") is None
