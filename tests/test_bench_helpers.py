"""Host logic of bench.py: the roofline arithmetic (algorithmic bytes and
flops per build, fractions of the peaks) and the clock-sampler summary that
decides whether a timed run saw throttling.  CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ST = {"n_quartets_kept": 133586661, "store_bytes": 602272832}   # stored_n200_m16 at tol 1e-10


def test_hbm_roofline_counts_the_algorithmic_bytes():
    """Split 16-bit store: kept unique quartets x 4 B + D in + J, K out
    (3 m N^2 doubles) = 549,706,644 B per build of stored_n200_m16."""
    r = bench.contraction_roofline("fp16x2", ST, 16, 200, 0.7e-3, {"fp64": 1.26, "fp32": 78.5})
    assert r["algorithmic_bytes"] == 133586661 * 4 + 3 * 16 * 200 * 200 * 8 == 549706644
    hbm, _, _ = bench.peaks()
    assert r["bound"] == "hbm" and r["peak"] == hbm
    assert r["achieved"] == pytest.approx(549706644 / 0.7e-3 / 1e9, abs=0.1)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm, abs=1e-4)
    assert r["kernel"] == "k_jk_umma"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alu_roofline_counts_twenty_m_flops_per_quartet(prec):
    """CUDA-core stores: 2 J + 8 K FMAs per density and kept unique quartet
    against the measured FMA rate of the precision."""
    peaks = {"fp64": 1.26, "fp32": 78.5}
    r = bench.contraction_roofline(prec, ST, 16, 200, 54.7e-3, peaks)
    assert r["algorithmic_flops"] == 133586661 * 20 * 16
    assert r["achieved"] == pytest.approx(133586661 * 20 * 16 / 54.7e-3 / 1e12, abs=1e-3)
    assert r["peak"] == peaks[prec] and r["bound"] == "alu" and r["kernel"] == "k_jk_cuda"


def test_double_fp32_peak_is_derived_from_the_fp32_rate():
    """Each double-FP32 product-add costs 12 FP32 instructions, so its peak
    is the FP32 FMA instruction rate / 12 x 2 flops."""
    r = bench.contraction_roofline("f32x2", ST, 16, 200, 17.5e-3, {"fp64": 1.26, "fp32": 78.47})
    assert r["peak"] == pytest.approx(78.47 / 12, abs=1e-3)
    assert r["traffic"] is None and "derived" in r["peak_source"]


def test_clock_summary_flags_throttling_and_skips_bad_lines():
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1100.0, Not Active, Not Active, Not Active, Active",
               "garbage",
               "[N/A], 2070, 1.0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.5, Active, Not Active, Not Active, Active"]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == 2055.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler(0).summary()
    assert empty == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
