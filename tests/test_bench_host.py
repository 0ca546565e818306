"""Host-side logic of bench.py that needs no GPU: the clock and throttle-reason summary."""

import bench


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.rows = [
        ["2070", "2070", "850.1", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1980", "2070", "1390.0", "Not Active", "Not Active", "Not Active", "Active"],
        ["2070", "2070", "900.0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"],
        ["2000"],  # a truncated line
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 5


def test_clock_summary_reports_every_slowdown_reason():
    c = bench.ClockSampler(0)
    c.rows = [["1200", "2070", "700", "Active", "Active", "Active", "Not Active"]]
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1200.0


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_forward_profile_figures_are_reported_only_for_the_captured_launch_shape():
    rec = bench.FORWARD_PROFILE.get((10_000_000, 16, 1))
    assert rec["traffic"] == 486.63e6 + 47.03e6 and rec["l1tex_pct"] == 93.1 and rec["lts_pct"] == 78.1
    assert bench.FORWARD_PROFILE.get((500_000, 16, 1)) is None
    assert bench.FORWARD_PROFILE.get((10_000_000, 32, 1)) is None


def test_peaks_come_from_the_measured_file_else_the_fallback(tmp_path):
    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6779.7, "bf16_tflops": 1944.1, "bf16_tflops_sustained": 1726.7}')
    assert bench.measured_peaks(str(f)) == (6779.7, 1944.1, "measured")
    assert bench.measured_peaks(str(tmp_path / "absent.json")) == (6800.0, 1900.0, "fallback")
    f.write_text('{"hbm_gbs": null}')
    assert bench.measured_peaks(str(f))[2] == "fallback"
