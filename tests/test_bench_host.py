"""Host-side work counts of bench.py, against the checker: the M2L pair
counts behind the tensor-core roofline and the near-field pair count behind
the reciprocal-square-root roofline, on a uniform and a clustered tree."""
import numpy as np
import pytest

import bench
from paper_1408_0210_gb300 import workloads as wl


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_m2l_pairs_equal_the_lists(orc, k):
    assert bench.m2l_pairs(k) == sum(len(orc.interaction_list(k, I)) for I in range(8 ** k))


@pytest.mark.parametrize("points,depth", [("uniform", 3), ("mixture", 4)])
def test_near_field_pairs_by_brute_force(orc, points, depth):
    x = wl.uniform_cube(3000, 61) if points == "uniform" else wl.gaussian_mixture(3000, 62)
    keys, outside = orc.morton_keys(x, [0.0, 0.0, 0.0], 1.0, depth)
    assert outside == 0
    _, off = orc.sort_leaves(keys, depth)
    cnt = np.diff(off)
    want = sum(int(cnt[I]) * sum(int(cnt[J]) for J in orc.neighbours(depth, I))
               for I in range(8 ** depth) if cnt[I]) - len(x)
    assert bench.near_field_pairs(off, depth) == want


def test_clock_summary_parses_the_sampler_lines():
    """The clock record of the timed region: median SM clock under load, the
    maximum, and which throttle reasons were ever active."""
    c = bench.ClockSampler(0)
    c.out = "\n".join([
        "0, 1965, 2070, 610.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ])
    s = c.summary()
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == 1965.0 and s["reasons"] == ["sw_power_cap"]
    c.out = ""
    assert c.summary() is None


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    """Roofline denominators: the measured file when present, else the
    recipe's fallback (6.8 TB/s, 1.9 PFLOP/s burst), labelled as such."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.peaks()
    assert p["source"] == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6696.5, "bf16_tflops": 1930.6}')
    p = bench.peaks()
    assert p["source"] == "measured" and p["hbm_gbs"] == 6696.5
