"""bench.py's roofline object (CPU, no GPU): the arithmetic that turns a
run's pixel-trials and loop time into achieved TFLOP/s, the fraction of the
peak, and the DRAM traffic per launch.

achieved = 9408 flop (2 x 48 filters x 49 taps, one multiply-add each way)
per pixel per trial / loop time; frac = achieved / peak; the FP32 form's
derived peak = SMs x 128 lanes x 2 flop x clock; traffic per launch = the
ncu bytes per pixel-trial x the pixel-trials of one launch (one persistent
launch per step), and none for per-trial or cluster launches."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(pix_trials, loop_ms, steps=5, cluster=1):
    return {"pix_trials": pix_trials, "loop_ms": loop_ms, "steps": steps, "cluster": cluster}


def test_fp32_roofline_arithmetic():
    npix = 24 * 512 * 512 + 24 * 256 * 256
    r = _run(pix_trials=5 * 2.4e9, loop_ms=5 * 480.0)
    rl = bench.roofline_of("fp32", "variant", r, npix, {"sms": 152, "ffma": 76.7}, 2070.0, loop_mode=2)
    achieved = 9408 * 2.4e9 / 0.480 / 1e12
    assert rl["achieved"] == pytest.approx(achieved, rel=1e-3)
    assert rl["peak"] == pytest.approx(76.7)
    assert rl["frac"] == pytest.approx(achieved / 76.7, abs=1e-4)
    assert rl["peak_derived"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12, rel=1e-4)
    assert rl["frac_of_derived"] == pytest.approx(achieved / rl["peak_derived"], abs=1e-4)
    assert rl["bound"] == "alu" and "MODE_PTRIAL" in rl["kernel"]
    bpt = bench.TRAFFIC_PER_PIXEL_TRIAL[("fp32", "variant")]
    assert 20.0 < bpt < 30.0  # about the 24 algorithmic bytes per pixel-trial
    assert rl["traffic"] == pytest.approx(bpt * 2.4e9, rel=1e-6)  # one launch = one step
    assert rl["traffic_per_full_batch_trial"] == pytest.approx(bpt * npix, rel=1e-6)
    # one trial over the whole batch: loop time / (pixel-trials / pixels)
    assert rl["ms_per_full_batch_trial"] == pytest.approx(5 * 480.0 / (5 * 2.4e9 / npix), rel=1e-4)


def test_no_traffic_for_per_trial_or_cluster_launches():
    npix = 1 << 20
    for mode, cluster in ((1, 1), (0, 1), (2, 4)):
        rl = bench.roofline_of("fp32", "variant", _run(1e9, 100.0, cluster=cluster), npix,
                               {"sms": 152, "ffma": 76.7}, 2070.0, loop_mode=mode)
        assert rl["traffic"] is None and rl["traffic_per_full_batch_trial"] is None
        assert "MODE_TRIAL" in rl["kernel"]


def test_fp32_peak_falls_back_to_unit_counts():
    rl = bench.roofline_of("fp32", "variant", _run(1e9, 100.0), 1 << 20, {"sms": 152}, 2070.0)
    assert rl["peak"] == pytest.approx(rl["peak_derived"])
    assert "unit counts" in rl["peak_basis"]


def test_tensor_forms_take_the_bf16_peak_and_the_tf32_ratio():
    sust, _ = bench.measured_bf16_sustained()
    r = _run(1e9, 100.0)
    bf = bench.roofline_of("bf16", "variant", r, 1 << 20, {"sms": 152}, 2070.0)
    br = bench.roofline_of("bf16r", "variant", r, 1 << 20, {"sms": 152}, 2070.0)
    tf = bench.roofline_of("tf32", "variant", r, 1 << 20, {"sms": 152}, 2070.0)
    assert bf["bound"] == br["bound"] == tf["bound"] == "tensor"
    assert bf["peak"] == pytest.approx(sust, abs=1e-3) and br["peak"] == bf["peak"]
    assert tf["peak"] == pytest.approx(sust * 1.1 / 2.25, abs=1e-3)  # dense TF32 / BF16 nominal ratio
    assert bf["achieved"] == tf["achieved"] == pytest.approx(9408 * 1e9 / 0.1 / 1e12, rel=1e-3)
    assert tf["frac"] == pytest.approx(tf["achieved"] / tf["peak"], abs=1e-4)
