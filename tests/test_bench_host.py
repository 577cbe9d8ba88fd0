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


def test_e2e_upload_bytes_match_what_setup_stages():
    """The e2e line declares what pc_sqa_setup copies host -> device: one
    16-bit coupling word per site and the 40 threshold words of every sweep
    (the anneal kernel's table row, [3 time counts][13 fields] + 1 pad)."""
    from paper_2503_10302_gb300 import build, pcomp
    build.build()
    for N, S in ((512, 10000), (64, 1), (4096, 30), (8, 0)):
        assert pcomp.pc_sqa_upload_bytes(N, S) == 2 * N + 40 * 4 * max(S, 1)
    assert pcomp.pc_sqa_upload_bytes(512, 10000) == 1601024


def test_alu_roofline_uses_twenty_ops_per_update():
    b = _bench()
    r = b._alu_roofline(1000.0, 40.0, "k")
    assert b.ALG_OPS_PER_FLIP == 20.0
    assert abs(r["achieved"] - 20.0) < 1e-12 and abs(r["frac"] - 0.5) < 1e-12
