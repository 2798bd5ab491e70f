"""Host-side logic of bench.py that needs no GPU: the clock-sample summary."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _line(t, sm, power, pcap="Not Active", hw="Not Active"):
    return f"2026/01/02 03:04:{t:06.3f}, 0, {sm}, 2070, {power}, 0x0, {hw}, Not Active, Not Active, {pcap}\n"


def test_clock_summary_keeps_the_timed_region():
    import bench
    lines = [_line(1.0, 1200, 150), _line(2.0, 2032, 900), _line(2.1, 2040, 950, pcap="Active"),
             _line(2.2, 2025, 940), _line(3.5, 1100, 140, hw="Active")]
    rows = bench.parse_clock_lines(lines)
    assert len(rows) == 5
    t0, t1 = rows[1]["ts"], rows[3]["ts"]
    s = bench.summarise_clocks(rows, (t0, t1))
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2032 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the region


def test_clock_summary_widens_a_short_region():
    import bench
    rows = bench.parse_clock_lines([_line(1.0, 2000, 800), _line(1.3, 2010, 820), _line(1.45, 2020, 810)])
    s = bench.summarise_clocks(rows, (rows[2]["ts"] - 0.01, rows[2]["ts"] + 0.01), slack=0.5)
    assert s["samples"] == 3 and s["window"].startswith("timed region +-")
    assert bench.summarise_clocks([], (0.0, 1.0)) is None
