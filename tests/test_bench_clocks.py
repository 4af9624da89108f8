"""Host logic of bench.py's clock record: nvidia-smi CSV samples are kept
only inside the timed region, throttle reasons are collected from them, and
a run without samples inside the region falls back to all of them."""
import datetime
import importlib.util
import os

_spec = importlib.util.spec_from_file_location(
    "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def _line(t, sm, smax, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, {smax}, 900.00, 0x0000000000000000, " + ", ".join(reasons) + "\n"


def test_samples_filtered_to_timed_region():
    t = 1.8e9
    lines = [_line(t - 1.0, 1000, 2070, ("Not Active", "Not Active", "Active", "Not Active")),
             _line(t + 0.05, 2070, 2070), _line(t + 0.10, 2055, 2070),
             _line(t + 0.15, 2070, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
             _line(t + 2.0, 900, 2070)]
    out = bench.parse_clock_samples(lines, t, t + 0.2)
    assert out["samples"] == 3 and out["samples_in_timed_region"] == 3
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]          # the thermal flag fell outside the region


def test_fallback_to_all_samples_and_garbage_lines():
    t = 1.8e9
    lines = ["", "garbage\n", _line(t - 5, 1500, 2070), _line(t - 4, 1700, 2070)]
    out = bench.parse_clock_samples(lines, t, t + 1)
    assert out["samples"] == 2 and out["samples_in_timed_region"] == 0
    assert out["sm_mhz"] == 1600
    assert bench.parse_clock_samples([], t, t + 1)["sm_mhz"] is None


def test_unparseable_timestamp_keeps_the_sample():
    lines = ["Tue Dec 3 20:13:52 2026, 0, 2070, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active\n"]
    out = bench.parse_clock_samples(lines, 0.0, 1.0)
    assert out["samples"] == 1 and out["samples_in_timed_region"] == 0 and out["sm_mhz"] == 2070
