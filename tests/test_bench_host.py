"""Host logic of bench.py on the CPU: the clock summary that decides whether
a timed run is accepted (median SM clock, maximum, throttle reasons seen
during the timed region), and the integer peak derived from the clock."""
import bench


def test_clock_summary_reasons_and_median():
    s = bench.ClockSampler(0)
    s.lines = [
        "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1200.5, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown():
    s = bench.ClockSampler(0)
    s.lines = ["1500, 2070, 1000, Not Active, Active, Not Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    out = bench.ClockSampler(0).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_alu_peak_follows_the_clock():
    assert bench.alu_peak_ops({}) == 152 * 4 * 16 * 2070e6
    assert bench.alu_peak_ops({"sm_max_mhz": 1000.0}) == 152 * 4 * 16 * 1e9
