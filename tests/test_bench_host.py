"""Host arithmetic of the benchmark's roofline entries (no GPU): the algorithmic
lane operations are the live units a launch processes times the operations per
unit, and the fraction is the achieved rate over the derived FP32 lane peak."""
import types

import pytest

import bench


def _problem():
    return types.SimpleNamespace(ne=128, npix=32400, nsub=16, nseg=64)


PEAKS = {"hbm_gbs": 6489.0, "sm_max_mhz": 2032.0}
PEAK = bench.lane_peak(148, {"sm_mhz": 1980.0}, PEAKS)


def test_lane_peak_uses_queried_sms_and_sampled_clock():
    rate, src = bench.lane_peak(148, {"sm_mhz": 1980.0}, PEAKS)
    assert rate == pytest.approx(148 * 128 * 1980e6)
    assert "148 SMs" in src and "1980 MHz" in src
    rate2, src2 = bench.lane_peak(160, None, PEAKS)        # no clock samples: the maximum clock
    assert rate2 == pytest.approx(160 * 128 * 2032e6) and "maximum" in src2


@pytest.mark.parametrize("stage", ["delays", "ray_adjoint"])
def test_ray_stage_counts_live_rays(stage):
    p = _problem()
    rays = 3_000_000                                     # live rays, not all ne * npix pairs
    ms, launches = 12.0, 20                              # 0.6 ms per launch
    r = bench.stage_roofline(stage, ms, launches, p, 402_718_720, PEAKS, rays, PEAK)
    ops = rays * (p.nseg + 1) * bench.OPS_PER_POINT[stage]
    assert r["algorithmic_ops"] == ops
    assert r["achieved"] == pytest.approx(ops / 0.6e-3 / 1e12)
    peak = 148 * 128 * 1980e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["bound"] == "alu" and "hbm" not in r
    # fewer live rays, proportionally less algorithmic work at the same time
    half = bench.stage_roofline(stage, ms, launches, p, 402_718_720, PEAKS, rays // 2, PEAK)
    assert half["frac"] == pytest.approx(r["frac"] / 2, rel=1e-6)


def test_gather_stage_counts_live_gathers_and_hbm_bytes():
    p = _problem()
    gathers = 433_783_322
    r = bench.stage_roofline("das_forward", 6.0, 10, p, 402_718_720, PEAKS, gathers, PEAK)
    assert r["algorithmic_ops"] == gathers * bench.OPS_PER_GATHER["das_forward"]
    nb = p.nsub * p.nsub
    bytes_ = 402_718_720 + p.ne * p.npix * 16 + nb * p.npix * 8
    assert r["hbm"]["algorithmic_bytes"] == bytes_
    assert r["hbm"]["achieved"] == pytest.approx(bytes_ / 0.6e-3 / 1e9)
    assert r["hbm"]["frac"] == pytest.approx(r["hbm"]["achieved"] / 6489.0)
    adj = bench.stage_roofline("das_adjoint", 6.0, 10, p, 402_718_720, PEAKS, gathers, PEAK)
    assert adj["hbm"]["algorithmic_bytes"] == bytes_ + p.ne * p.npix * 4


def test_lane_peak_prefers_the_measured_rate():
    rate, src = bench.lane_peak(148, {"sm_mhz": 2032.0}, PEAKS, measured=36.0e12)
    assert rate == 36.0e12
    assert src.startswith("measured") and "0.935" in src


def test_interval_stats_of_kernel_traces():
    """Busy-time sweep of the batch trace: hand-made intervals with known answers."""
    # [0, 4] and [2, 6] overlap on [2, 4]; [8, 10] after an idle gap [6, 8]
    st = bench.interval_stats([(0.0, 4.0), (2.0, 6.0), (8.0, 10.0)])
    assert st["span"] == 10.0
    assert abs(st["idle_fraction"] - 0.2) < 1e-12                 # [6, 8]
    assert abs(st["single_kernel_fraction"] - 0.6) < 1e-12        # [0, 2], [4, 6], [8, 10]
    assert abs(st["mean_kernels_in_flight"] - 1.0) < 1e-12        # (4 + 4 + 2) / 10
    # nested and touching intervals
    st = bench.interval_stats([(0.0, 10.0), (1.0, 2.0), (2.0, 3.0)])
    assert st["idle_fraction"] == 0.0 and abs(st["single_kernel_fraction"] - 0.8) < 1e-12
    assert bench.interval_stats([])["span"] == 0.0
