"""bench.py's host-side arithmetic on CPU: the roofline object (achieved rate per launch), the
projection rates, the clock summary, the peak file, and the oracle's step timed in units (the
unit cycle must reproduce the oracle's own HOOI and MP passes)."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from oracle import tucker_oracle as O  # noqa: E402
from paper_0711_2023_gb300 import synth  # noqa: E402


def test_roofline_of():
    # 4 launches of 2 TFLOP each in 8 ms total: 2e12 / 2e-3 s = 1000 TFLOP/s per launch
    prof = {"k": {"launches": 4, "ms": 8.0, "flops": 8e12, "bytes": 4e9}}
    r = bench.roofline_of(prof, "k", 16.0, "tensor", 2000.0, "TFLOP/s", "test")
    assert math.isclose(r["achieved"], 1000.0) and math.isclose(r["frac"], 0.5)
    assert math.isclose(r["share_of_step"], 0.5) and r["launches"] == 4
    assert r["traffic"] is None
    assert math.isclose(r["algorithmic_bytes"], 1e9)
    assert bench.roofline_of(prof, "missing", 16.0, "alu", 1.0, "TFLOP/s", "t") is None
    t = bench.roofline_of(prof, "k", 16.0, "tensor", 2000.0, "TFLOP/s", "t", traffic=1.5e9)
    assert t["traffic"] == 1.5e9


def test_ttmc_rates():
    prof = {"ttmc_mixed": {"launches": 10, "ms": 5.0, "flops": 5e10, "bytes": 1e9}}
    r = bench.ttmc_rates(prof, "ttmc_mixed", 80.0, 8000.0, "n")
    assert math.isclose(r["algorithmic_gbs"], 200.0) and math.isclose(r["frac_hbm"], 0.025)
    assert math.isclose(r["tflops"], 10.0) and math.isclose(r["frac_alu"], 0.125)
    assert math.isclose(r["ms_per_launch"], 0.5)
    assert bench.ttmc_rates({}, "ttmc_mixed", 80.0, 8000.0, "n") is None


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


def test_estimate_step_seconds():
    times = {u: [] for u in bench.REFERENCE_UNITS}
    for i, u in enumerate(bench.REFERENCE_UNITS):
        times[u] = [1.0 + i, 3.0 + i]              # mean 2 + i
    s, missing = bench.estimate_step_seconds(times)
    assert math.isclose(s, sum(2.0 + i for i in range(10))) and missing == []
    part = {u: ([2.0] if i < 4 else []) for i, u in enumerate(bench.REFERENCE_UNITS)}
    s, missing = bench.estimate_step_seconds(part)
    assert math.isclose(s, 20.0) and len(missing) == 6


def test_unit_cycle_reproduces_the_oracle_passes(monkeypatch):
    # The ten units, run in order, are exactly one HOOI pass and one MP pass from the start.
    monkeypatch.setattr(bench, "CORE", (4, 3, 5))
    X = synth.random_sparse_tensor((12, 10, 9), 300, synth.config_seed(77))
    start = bench.oracle_start(X, None, None)
    st = bench.OracleStep(X, start)
    for u in bench.REFERENCE_UNITS:
        st.run(u)
    h = O.hooi(X.dims, X.idx, X.val, (4, 3, 5), -np.inf, 1, init=start)
    m = O.mp(X.dims, X.idx, X.val, (4, 3, 5), -np.inf, 1, init=start)
    assert abs(st.fits["hooi"] - h["fit"]) <= 1e-14
    assert abs(st.fits["mp"] - m["fit"]) <= 1e-14
    # the MP start given explicitly equals the pseudo HO-SVD start (same leading eigenvectors)
    m0 = O.mp(X.dims, X.idx, X.val, (4, 3, 5), -np.inf, 1)
    assert abs(m0["fit"] - m["fit"]) <= 1e-12
