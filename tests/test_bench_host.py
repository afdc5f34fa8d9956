"""Host logic of the benchmark (CPU only): the algorithmic byte count of the
level-0 launch, the hash guard on the captured DRAM traffic, the clock
sampler's summary of nvidia-smi lines, the workload configuration and the
fallback peaks."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_level0_algorithmic_bytes_by_hand():
    """8 x 4 frame, 5 disoccluded pixels: 29 spatial logits, L^0, W_t L_{t-1},
    mask and both outputs on every pixel, 25 temporal logits on the 27 others,
    12 B per pixel of the 4 x 2 coarse level."""
    W, H = 8, 4
    mask = np.zeros((H, W), np.uint8)
    mask.flat[[0, 3, 9, 17, 31]] = 1
    per_pixel = 29 * 4 + 12 + 12 + 1 + 24
    expect = 32 * per_pixel + 27 * 25 * 4 + 8 * 12
    assert bench.level0_algorithmic_bytes(W, H, mask) == expect


def test_level0_bytes_at_1080p_match_the_documented_figure():
    """About 545 MB per 1080p launch with 5 % of the pixels disoccluded."""
    W, H = 1920, 1080
    mask = np.zeros((H, W), np.uint8)
    mask.flat[: int(0.05 * W * H)] = 1
    b = bench.level0_algorithmic_bytes(W, H, mask)
    assert 544e6 < b < 546e6


def test_traffic_guard(monkeypatch):
    t = dict(bench.LEVEL0_TRAFFIC)
    assert bench.level0_traffic("4k") is None            # captured on 1080p only
    got = bench.level0_traffic("1080p")
    assert got in (None, t["bytes_per_launch"])          # None once the sources change
    monkeypatch.setitem(bench.LEVEL0_TRAFFIC, "sha256", "0" * 64)
    assert bench.level0_traffic("1080p") is None


def test_traffic_guard_hashes_every_listed_source():
    for f in bench.LEVEL0_TRAFFIC["sources"]:
        assert os.path.exists(os.path.join(ROOT, f)), f


def _line(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"2026/01/01 00:00:00.000, {sm}, {smax}, 900.0, 0x0, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout: 0})()
    cs.t_start, cs.t_end = 10.0, 20.0
    cs.lines = [(9.0, _line(1000, 2070)),                        # before the region
                (11.0, _line(2070, 2070)), (12.0, _line(2055, 2070, cap="Active")),
                (13.0, _line(2070, 2070)), (19.9, _line(1980, 2070)),
                (25.0, _line(500, 2070, hwt="Active"))]          # after the region
    out = cs.stop()
    assert out["sm_mhz"] == pytest.approx(2062.5)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 4


def test_clock_summary_short_region_takes_the_next_samples():
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout: 0})()
    cs.t_start, cs.t_end = 10.0, 10.01
    cs.lines = [(10.5, _line(2070, 2070, hw="Active")), (10.6, _line(2070, 2070)),
                (10.7, _line(1500, 2070))]
    out = cs.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown"]


def test_clock_summary_reads_the_tail_of_the_same_load():
    """A short timed region is followed by a tail of the same steps: the
    samples of both count, later ones do not."""
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout: 0})()
    cs.t_start, cs.t_end, cs.t_tail_end = 10.0, 10.004, 10.5
    cs.lines = [(9.9, _line(900, 2070)), (10.05, _line(2070, 2070)),
                (10.3, _line(2055, 2070)), (10.49, _line(2070, 2070)),
                (11.0, _line(600, 2070, hwt="Active"))]
    out = cs.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    assert out["window_s"] == pytest.approx(0.5)


def test_clock_summary_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_workload_config_names_the_workload():
    for name, (W, H, F, B, L) in bench.WORKLOADS.items():
        c = bench.workload_config(name)
        assert c["W"] == W and c["H"] == H and c["frames"] == F and c["spp"] == B
        assert f"{W}x{H}" in c["workload"] and "model" not in c
        json.dumps(c)


def test_measured_peaks_or_fallback(tmp_path, monkeypatch):
    peaks, kind = bench.measured_peaks()
    assert kind in ("measured", "fallback") and peaks["hbm_gbs"] > 0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks == {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def test_reference_band_scales_with_the_step_count():
    """The reference arm's per-step band shrinks as the step count grows so
    that the run stays near its time target, within [2^(L-1), H/8] rows."""
    W, H, L = 1920, 1080, 3
    spp = 0.164 / (1920 * 132)  # seconds per pixel of the FP64 oracle, one core
    assert bench.reference_band_rows(W, H, L, 20, spp) == 132          # the whole band
    r = bench.reference_band_rows(W, H, L, 2000, spp)
    assert r % 4 == 0 and bench.REFERENCE_MIN_ROWS <= r < 132
    assert 2000 * r * W * spp <= bench.REFERENCE_SECONDS
    assert bench.reference_band_rows(W, H, L, 10 ** 7, spp) == bench.REFERENCE_MIN_ROWS
    assert bench.reference_band_rows(64, 64, 2, 1, 1e-9) == 8          # H/8 for a small frame
    assert bench.reference_band_rows(64, 64, 2, 10 ** 7, 1e-3) == 8    # the floor capped at H/8
