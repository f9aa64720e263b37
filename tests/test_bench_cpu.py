"""bench.py's host-side arithmetic on CPU: the roofline object (achieved rate per launch, the
ncu-derived traffic), the TTMc rates, the clock summary and the peak file."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_of():
    # 4 launches of 2 TFLOP each in 8 ms total: 2e12 / 2e-3 s = 1000 TFLOP/s per launch
    prof = {"k": {"launches": 4, "ms": 8.0, "flops": 8e12, "bytes": 4e9}}
    r = bench.roofline_of(prof, "k", 16.0, "tensor", 2000.0, "TFLOP/s", "test")
    assert math.isclose(r["achieved"], 1000.0) and math.isclose(r["frac"], 0.5)
    assert math.isclose(r["share_of_step"], 0.5) and r["launches"] == 4
    assert r["traffic"] is None                       # no ncu ratio for this kernel
    assert bench.roofline_of(prof, "missing", 16.0, "alu", 1.0, "TFLOP/s", "t") is None
    # GB/s roof from bytes
    g = bench.roofline_of(prof, "k", 16.0, "hbm", 1000.0, "GB/s", "t", per="bytes")
    assert math.isclose(g["achieved"], 500.0)         # 1e9 B / 2e-3 s


def test_ncu_traffic_ratio():
    # traffic per launch = (ncu DRAM bytes / algorithmic bytes of the capture) x algorithmic bytes
    assert 0.8 < bench.NCU_TRAFFIC_RATIO["syrk_f64"] < 1.1
    assert 1.0 <= bench.NCU_TRAFFIC_RATIO["gram_bf16x3"] < 1.2
    prof = {"syrk_f64": {"launches": 2, "ms": 2.0, "flops": 2e9, "bytes": 2e8}}
    r = bench.roofline_of(prof, "syrk_f64", 4.0, "alu", 1.25, "TFLOP/s", "t")
    assert math.isclose(r["traffic"], bench.NCU_TRAFFIC_RATIO["syrk_f64"] * 1e8)
    assert math.isclose(r["algorithmic_bytes"], 1e8)


def test_ttmc_rates():
    prof = {"ttmc_mixed": {"launches": 10, "ms": 5.0, "flops": 5e10, "bytes": 1e9}}
    r = bench.ttmc_rates(prof, "ttmc_mixed", 80.0, 8000.0)
    assert math.isclose(r["algorithmic_gbs"], 200.0) and math.isclose(r["frac_hbm"], 0.025)
    assert math.isclose(r["tflops"], 10.0) and math.isclose(r["frac_alu"], 0.125)
    assert math.isclose(r["ms_per_launch"], 0.5)
    assert bench.ttmc_rates({}, "ttmc_mixed", 80.0, 8000.0) is None


def test_parse_clocks():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2010, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1990, 2070, 1395.2, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clocks(lines)
    assert c["sm_mhz"] == 2010 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.parse_clocks([]) is None


def test_load_peaks_reads_measured_file():
    peaks, src = bench.load_peaks()
    assert src in ("measured", "fallback")
    assert peaks["hbm_gbs"] > 1000 and peaks["bf16_tflops"] > 100
