"""Host logic of bench.py that needs no GPU: the clock and throttle-reason
summary taken from nvidia-smi samples during the timed region."""
import bench

IDLE = "2070, 2070, 950.12, 0x0000000000000000, Not Active, Not Active, " \
       "Not Active, Not Active"


def line(sm, reasons=()):
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
             "sw_power_cap")
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([str(sm), "2070", "1200.5", "0x4"] + flags)


def test_median_clock_and_no_reasons():
    out = bench.parse_clock_lines([line(2070), line(2055), line(1980)])
    assert out == {"sm_mhz": 2055, "sm_max_mhz": 2070.0, "reasons": [],
                   "samples": 3}
    assert bench.parse_clock_lines([IDLE])["reasons"] == []


def test_every_active_reason_is_reported_once():
    out = bench.parse_clock_lines([
        line(1900, ("sw_power_cap",)), line(1850, ("hw_slowdown",)),
        line(1870, ("sw_power_cap", "sw_thermal_slowdown"))])
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap",
                              "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1870


def test_malformed_and_unavailable_samples_are_skipped():
    out = bench.parse_clock_lines([
        "", "clocks.current.sm [MHz], clocks.max.sm [MHz]",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        line(2070)])
    assert out["samples"] == 1 and out["sm_mhz"] == 2070
    assert bench.parse_clock_lines([])["sm_mhz"] is None
