"""bench.py's reading of the clock samples taken during the timed region (no GPU): the median
SM clock, the maximum, and every throttle reason that was active in any sample."""
import bench


def line(sm, smax=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 1190.25, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_median_max_and_no_reasons():
    r = bench.parse_clock_lines([line(2070), line(1965), line(2070), line(2040)])
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}


def test_each_reason_is_reported_once():
    lines = [line(2070), line(1800, cap="Active"), line(1700, cap="Active"),
             line(1500, hw="Active"), line(1400, hwt="Active", swt="Active")]
    r = bench.parse_clock_lines(lines)
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                            "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1700.0 and r["samples"] == 5


def test_unparsable_lines_are_skipped_but_their_reasons_count():
    lines = ["", "garbage", "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Active",
             line(2070), "0, 2070, 2070"]
    r = bench.parse_clock_lines(lines)
    assert r["samples"] == 1 and r["sm_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]     # a throttle flag is never hidden


def test_no_samples():
    assert bench.parse_clock_lines([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                           "samples": 0}


def test_sampler_without_nvidia_smi_reports_it():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
