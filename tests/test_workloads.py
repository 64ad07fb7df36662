"""The seeded input recipes: shapes, ranges, orders and determinism."""
import numpy as np

from paper_1408_0210_gb300 import workloads as wl


def test_points_shapes_ranges_and_seeds():
    x = wl.uniform_cube(10000, 1)
    assert x.shape == (10000, 3) and x.dtype == np.float64
    assert (x >= 0).all() and (x < 1).all()
    assert np.array_equal(x, wl.uniform_cube(10000, 1)) and not np.array_equal(x, wl.uniform_cube(10000, 2))
    assert abs(x.mean() - 0.5) < 0.01
    g = wl.gaussian_mixture(20000, 3)
    assert (g >= 0).all() and (g <= 1).all()
    # 8 tight clusters: far more mass in the densest 1% of leaves than uniform
    h, _ = np.histogramdd(g, bins=16, range=[(0, 1)] * 3)
    top = np.sort(h.ravel())[::-1][:41].sum() / len(g)
    assert top > 0.3


def test_potentials_layout_and_law():
    s = wl.sigma_uniform(5000, 4, 7)
    assert s.shape == (5000, 4) and s.flags.f_contiguous
    assert (np.abs(s) <= 1).all() and abs(s.mean()) < 0.05
    assert np.array_equal(s, wl.sigma_uniform(5000, 4, 7))
    n = wl.sigma_normal(20000, 2, 8)
    assert n.flags.f_contiguous and abs(n.std() - 1.0) < 0.02


def test_batch_sizes_and_samples():
    b = wl.batch_sizes(32, 16384, 262144, 40)
    assert len(b) == 32 and min(b) >= 16384 and max(b) <= 262144
    t = wl.sample_targets(1000, 200, 5)
    assert len(t) == 200 and len(np.unique(t)) == 200 and (np.diff(t) > 0).all()
    assert t.min() >= 0 and t.max() < 1000
    assert len(wl.sample_targets(50, 200, 5)) == 50
