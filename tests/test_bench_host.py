"""Host logic of bench.py (no GPU): the clock and throttle-reason summary."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_median_max_and_reasons():
    S = _bench().ClockSampler.summarize
    lines = [
        "0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = S(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_is_none():
    S = _bench().ClockSampler.summarize
    assert S([]) is None
    assert S(["not, enough, fields"]) is None
