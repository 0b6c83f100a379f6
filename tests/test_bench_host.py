"""Host-side pieces of the benchmark on CPU: the clock record's summary (throttle reasons that
reject a run), the single-rank job rate, the H_eff flop count against a direct count."""
import sys

import numpy as np

from tests.conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(sm, mx, *reasons):
    flags = ["Active" if r else "Not Active" for r in reasons]
    return [x.strip() for x in f"0, {sm}, {mx}, 812.3, 0x0, {', '.join(flags)}".split(",")]


def test_clock_summary_reasons_and_median():
    s = bench.ClockSampler(0)
    s.rows = [_row(2070, 2070, 0, 0, 0, 0), _row(2055, 2070, 0, 0, 0, 1), _row(2070, 2070, 0, 0, 0, 0)]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.rows.append(_row(1500, 2070, 1, 0, 1, 0))
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]


def test_single_rank_rate_and_heff_flops():
    assert bench.whole_job_rate(1, 10.0, 4.0) == 2.5
    # 8 d^2 chi_l chi_r (w_l chi_l + w_r chi_r): count the two GEMMs of the contraction directly
    chi_l, chi_r, d, wl, wr = 5, 7, 3, 4, 6
    first = wl * chi_l * (d * d * chi_r) * chi_l          # L (w_l chi_l x chi_l) times theta
    last = (chi_l * d * d) * chi_r * (chi_r * wr)         # T3 times R, summed over channels
    assert bench.heff_flops(chi_l, chi_r, d, wl, wr) == 8 * (first + last)
    assert np.isclose(bench.heff_flops(128, 128, 8, 24, 24), 5.15e10, rtol=1e-2)  # split middle bond
