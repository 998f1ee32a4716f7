"""Host-side pieces of bench.py (no GPU): the FFT work count, the grid size
rule it shares with the library, and the roofline entry of a traced slot."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from synth import make_system  # noqa: E402


def test_smooth_grid_sizes():
    # the smallest 2^a 3^b 5^c at or above n (the library's FFT grid rule)
    assert [bench._smooth(n) for n in (1, 17, 41, 45, 47, 49, 53, 57, 73)] == [1, 18, 45, 45, 48, 50, 54, 60, 75]


def test_fft_work_scales_with_states_and_undercuts_the_direct_sum():
    s = make_system("h2_6000", with_amat=False)
    fl, by = bench.fft_work(s)
    s2 = dict(s, n_s=2 * int(s["n_s"]))
    fl2, by2 = bench.fft_work(s2)
    assert abs(fl2 / fl - 2.0) < 1e-12 and abs(by2 / by - 2.0) < 1e-12
    ng = int(s["n_g"][0])
    direct = 8.0 * ng * ng * int(s["n_s"])
    assert 10 * fl < direct


def test_roofline_entry_of_the_series():
    s = make_system("tiny400", with_amat=False)
    tr = {"chebyshev_series": [0.5, 10]}  # 10 launches, 0.05 ms each
    roof = bench.roofline_of("chebyshev_series", tr, s, "fp32+fft", 14)
    fl, _ = bench.algorithmic_work("chebyshev_series", s, "fp32", 14)
    assert roof["bound"] == "alu" and roof["peak"] == bench.FP64_PEAK_TFLOPS
    assert np.isclose(roof["achieved"], fl / 0.05e-3 / 1e12)
    assert np.isclose(roof["frac"], roof["achieved"] / roof["peak"])
    assert roof["traffic"] is None  # no capture for this workload


def test_roofline_entry_of_the_fft_slot():
    s = make_system("h2_6000", with_amat=False)
    tr = {"fft_interstitial": [0.3, 10]}  # 0.03 ms per step
    roof = bench.roofline_of("fft_interstitial", tr, s, "fp32+fft", 14)
    fl, _ = bench.fft_work(s)
    assert roof["bound"] == "alu"
    assert np.isclose(roof["peak"], bench.SM_COUNT * bench.FP32_LANES * 2 * bench.SM_MAX_MHZ * 1e6 / 1e12)
    assert np.isclose(roof["achieved"], fl / 0.03e-3 / 1e12)
    roof64 = bench.roofline_of("fft_interstitial", tr, s, "fp64+fft", 14)
    assert roof64["peak"] == bench.FP64_PEAK_TFLOPS


def test_density_feedback_is_not_sharded():
    """A k-point shard or subset of a density-feedback run would feed back a
    partial density: the benchmark refuses it before any GPU work; the forms
    without feedback shard freely."""
    assert bench.shard_refusal("fp64+fft+hartree", 2, "") is not None
    assert bench.shard_refusal("fp32+fft+hartree", 1, "0,1") is not None
    assert bench.shard_refusal("fp64+fft+hartree", 1, "") is None
    for form in ("fp64", "bf16x3", "fp32+fft+dv"):
        assert bench.shard_refusal(form, 8, "0,1") is None
