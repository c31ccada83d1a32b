"""Host-side logic of the benchmark that needs no GPU: the clock samples kept
for the timed region, the algorithmic bytes of the stage kernel, and the
per-workload lookup of the committed ncu traffic."""
import datetime
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(ts, dev, sm, smax, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([stamp, str(dev), str(sm), str(smax), "900.0", "0x0"] + flags) + "\n"


def test_clock_samples_inside_the_timed_window(tmp_path):
    t0 = 1_800_000_000.0
    p = tmp_path / "clk.csv"
    p.write_text(_line(t0 - 0.2, 0, 1200, 2070, ["hw_slowdown"])  # before the window: ignored
                 + _line(t0 + 0.05, 0, 2070, 2070)
                 + _line(t0 + 0.10, 1, 900, 2070)  # another GPU: ignored
                 + _line(t0 + 0.15, 0, 2050, 2070, ["sw_power_cap"])
                 + _line(t0 + 0.25, 0, 2070, 2070)
                 + _line(t0 + 0.60, 0, 1000, 2070, ["hw_thermal_slowdown"]))  # after: ignored
    out = bench.parse_clock_samples(str(p), 0, t0, t0 + 0.3)
    assert out["samples"] == 3 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_samples_fall_back_to_all_when_none_is_inside(tmp_path):
    t0 = 1_800_000_000.0
    p = tmp_path / "clk.csv"
    p.write_text(_line(t0 - 1.0, 0, 2000, 2070) + _line(t0 + 2.0, 0, 1900, 2070, ["hw_slowdown"]))
    out = bench.parse_clock_samples(str(p), 0, t0, t0 + 0.001)
    assert out["samples"] == 2 and out["window"] == "around the timed region"
    assert out["reasons"] == ["hw_slowdown"]
    assert bench.parse_clock_samples(str(p), 3, t0, t0 + 1.0) is None  # no sample of that GPU


def test_stage_bytes_per_cell():
    # Euler P2: u^(i-1) read and u^(i) written (96 B each), u^n read in stages 2-3,
    # 13 geometry words, 3 neighbour ids + packed faces, 7 record words + 3 slots
    s = 4
    S = 24 * s
    per_stage = 2 * S + 13 * s + 12 + 1 + 10 * s
    assert bench.stage_bytes_per_cell(True) == pytest.approx((3 * per_stage + 2 * S) / 3)
    assert bench.stage_bytes_per_cell(True) == pytest.approx(361.0)


def test_traffic_lookup_is_per_workload_and_hash_checked():
    h = bench.kernel_hash()
    assert bench.read_traffic("0" * 16, "dmr") is None  # another kernel source
    assert bench.read_traffic(h, "no-such-workload") is None
    v = bench.read_traffic(h, "dmr")
    assert v is None or v > 0
