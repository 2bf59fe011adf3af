"""Host logic of bench.py (no GPU): the committed DRAM traffic figure is used
only for the workload and kernel source it was captured on, and the clock
record keeps every throttle reason seen during the timed region."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _committed_traffic():
    rows = {}
    with open(os.path.join(ROOT, "profiles", "k2_spmv_traffic.txt")) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                rows[k.strip()] = v.strip()
    return rows


def test_traffic_follows_workload_and_kernel_source(monkeypatch):
    rows = _committed_traffic()
    wl = rows["workload"]
    if rows["kernel_source_sha256_16"] == bench.kernel_source_hash():
        assert bench.profiled_traffic(wl) == float(rows["dram_bytes_per_launch"])
        # taken at one column-block count: another count drops it
        assert bench.profiled_traffic(wl, int(rows["col_blocks"])) == float(rows["dram_bytes_per_launch"])
        assert bench.profiled_traffic(wl, int(rows["col_blocks"]) + 1) is None
    else:
        assert bench.profiled_traffic(wl) is None
    assert bench.profiled_traffic("rmat_s16") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic(wl) is None  # a changed kernel drops the stale figure


def test_clock_summary():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = bench.ClockSampler.summarize([ok, ok, capped, "garbage", "0, N/A, 2070, 1, 0, a, b, c, d"])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.ClockSampler.summarize([ok, hot, capped])
    assert s["sm_mhz"] == 1980.0 and s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarize([])["reasons"] == ["no samples"]
