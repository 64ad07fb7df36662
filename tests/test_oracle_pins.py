"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check ties an oracle function to something independent of it: values
computed by hand, closed forms, brute force on tiny inputs, the interpolation
property of Section 2 (Property 2.1), exactness on separable low-rank kernels,
the structural facts of the tree and lists (Sections 3.2-3.3) and the
convergence of the method as the EIM tolerance shrinks.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1408_0210_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# O1, Eq. (1)
# --------------------------------------------------------------------------
def test_direct_sum_hand_example(orc):
    g = json.load(open(os.path.join(GOLD, "direct_sum_hand.json")))
    x = np.array(g["points"])
    f = orc.direct_sum("inv_r", x, x, np.array(g["sigma"]))[:, 0]
    np.testing.assert_allclose(f, g["f"], rtol=1e-15, atol=0)


def test_kernels_hand_values(orc):
    """Every transcendental kernel branch of the oracle against its closed form
    at points worked out by hand (tests/golden/kernels_hand.json; written by
    make_kernels_hand.py from those closed forms alone).  The anisotropic
    kernel is checked with the same |z| along each axis, so the 0.01 weight
    on the second component is pinned to that axis."""
    g = json.load(open(os.path.join(GOLD, "kernels_hand.json")))
    seen = set()
    for c in g["cases"]:
        v = orc.kernel(c["kernel"], np.array([c["z"]]))[0]
        assert abs(v - c["k"]) <= 1e-15 * abs(c["k"]), (c["kernel"], c["z"], v, c["k"])
        seen.add(c["kernel"])
    assert seen == {"config3", "exp_r2", "cos20r_r", "sqrt_r2p1"}
    # a weight on another axis would change the value by orders of magnitude
    by_z = {tuple(c["z"]): c["k"] for c in g["cases"] if c["kernel"] == "config3"}
    assert by_z[(0.0, 10.0, 0.0)] > 9 * by_z[(10.0, 0.0, 0.0)]


def test_direct_sum_closed_forms(orc):
    x = wl.uniform_cube(700, 11)
    y = wl.uniform_cube(500, 12)
    s = wl.sigma_uniform(500, 2, 13)
    # K = 1: f_i = sum_j sigma_j
    f = orc.direct_sum("one", x, y, s, exclude_self=False)
    np.testing.assert_allclose(f, np.tile(s.sum(0), (700, 1)), rtol=1e-12)
    # K = |x - y|^2 = |x|^2 S0 - 2 x.S1 + S2 with moments of the sources
    f = orc.direct_sum("quad", x, y, s, exclude_self=False)
    S0, S1, S2 = s.sum(0), y.T @ s, ((y * y).sum(1)) @ s
    ref = (x * x).sum(1)[:, None] * S0 - 2 * x @ S1 + S2
    np.testing.assert_allclose(f, ref, rtol=1e-11)
    # self exclusion: sets coincide, K = 1 gives S - sigma_i
    f = orc.direct_sum("one", y, y, s, exclude_self=True)
    np.testing.assert_allclose(f, s.sum(0) - s, rtol=1e-12, atol=1e-12)


def test_direct_sum_shell_potential(orc):
    # every point of a sphere of radius a is at distance a from its centre
    n = 2000
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    a = 0.37
    c = np.array([0.5, 0.5, 0.5])
    pts = c + a * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    s = wl.sigma_uniform(n, 1, 5)
    f = orc.direct_sum("inv_r", c[None], pts, s, exclude_self=False)
    assert abs(f[0, 0] - s.sum() / a) <= 1e-12 * np.abs(s).sum() / a


def test_direct_sum_summation_accuracy_and_subset(orc):
    x = wl.uniform_cube(4096, 1)
    s = wl.sigma_uniform(4096, 1, 101)
    f = orc.direct_sum("inv_r", x, x, s)
    fl = orc.direct_sum("inv_r", x, x, s, long_double=True)
    assert np.linalg.norm(f - fl) / np.linalg.norm(fl) < 1e-13
    idx = wl.sample_targets(4096, 100, 7)
    fs = orc.direct_sum("inv_r", x, x, s, tgt_idx=idx)
    np.testing.assert_array_equal(fs, f[idx])


# --------------------------------------------------------------------------
# Tree (Section 3.3)
# --------------------------------------------------------------------------
def _morton_py(ix, iy, iz, depth):
    key = 0
    for b in range(depth):
        key |= ((ix >> b) & 1) << (3 * b)
        key |= ((iy >> b) & 1) << (3 * b + 1)
        key |= ((iz >> b) & 1) << (3 * b + 2)
    return key


@pytest.mark.parametrize("depth", [1, 3, 5])
def test_morton_keys_exact(orc, depth):
    x = wl.uniform_cube(3000, 21 + depth)
    x[0] = [1.0, 0.0, 1.0]          # upper faces clamp into the last box
    x[1] = [0.5, 0.25, 0.125]       # exactly on box boundaries
    keys, outside = orc.morton_keys(x, [0.0, 0.0, 0.0], 1.0, depth)
    assert outside == 0
    n = 1 << depth
    for i in range(len(x)):
        c = [min(n - 1, int(math.floor(Fraction(v) * n))) for v in x[i]]
        assert keys[i] == _morton_py(*c, depth)


def test_morton_keys_general_box_and_outside(orc):
    lo = np.array([-0.5, 2.0, 10.0])
    L = 2.0
    x = lo + L * wl.uniform_cube(500, 3)
    x[0, 0] = lo[0] - 1e-9
    x[1, 2] = lo[2] + L + 1e-9
    keys, outside = orc.morton_keys(x, lo, L, 4)
    assert outside == 2
    for i in range(2, len(x)):
        t = [(Fraction(x[i, a]) - Fraction(lo[a])) * Fraction(16) / Fraction(L) for a in range(3)]
        c = [min(15, int(math.floor(v))) for v in t]
        # FP64 rounding of (x - lo) * 2^k / L can cross an integer only when
        # the exact value lies within a few ulps of it
        near_int = any(abs(float(v - round(v))) < 1e-12 for v in t)
        assert keys[i] == _morton_py(*c, 4) or near_int


def test_sort_is_stable_and_offsets(orc):
    x = wl.gaussian_mixture(5000, 3)
    keys, _ = orc.morton_keys(x, [0, 0, 0], 1.0, 4)
    perm, off = orc.sort_leaves(keys, 4)
    order = np.lexsort((np.arange(len(keys)), keys))
    np.testing.assert_array_equal(perm, order)
    counts = np.bincount(keys, minlength=8 ** 4)
    np.testing.assert_array_equal(np.diff(off), counts)
    assert off[0] == 0 and off[-1] == len(x)


# --------------------------------------------------------------------------
# Neighbourhood and interaction lists (Sections 3.2, 3.3.2)
# --------------------------------------------------------------------------
def _coords(level):
    n = 1 << level
    c = np.array([[i, j, k] for k in range(n) for j in range(n) for i in range(n)])
    keys = np.array([_morton_py(*t, level) for t in c])
    out = np.zeros_like(c)
    out[keys] = c
    return out


@pytest.mark.parametrize("level", [2, 3])
def test_interaction_list_brute_force(orc, level):
    c = _coords(level)
    nbox = len(c)
    total = 0
    for I in range(nbox):
        got = sorted(orc.interaction_list(level, I))
        par = c[I] >> 1
        exp = [J for J in range(nbox)
               if np.abs((c[J] >> 1) - par).max() <= 1 and np.abs(c[J] - c[I]).max() > 1]
        assert got == exp
        total += len(got)
    assert total == {2: 3096, 3: 53352}[level]


def test_list_sizes_match_the_separable_count(orc):
    """Section 3.3 lists at full levels against a closed form: per dimension
    a box at index i has the children of its parent's neighbours,
    [2(i//2) - 2, 2(i//2) + 3] clipped to the grid, of which its own
    neighbours [i - 1, i + 1] are excluded, so the number of (I, J) pairs of a
    level is (sum of the first counts)^3 - (sum of the second)^3, and the near
    (leaf, neighbour) pairs are (3n - 2)^3."""
    for k in (2, 3, 4, 5):
        n = 1 << k
        sa = sum(min(n - 1, 2 * (i // 2) + 3) - max(0, 2 * (i // 2) - 2) + 1 for i in range(n))
        sb = sum(min(n - 1, i + 1) - max(0, i - 1) + 1 for i in range(n))
        got = sum(len(orc.interaction_list(k, I)) for I in range(8 ** k))
        assert got == sa ** 3 - sb ** 3
        assert sum(len(orc.neighbours(k, I)) for I in range(8 ** k)) == (3 * n - 2) ** 3
    # all far-field levels of a full depth-5 tree: 6,039,504 M2L pairs
    assert sum(len(orc.interaction_list(k, I)) for k in (2, 3, 4, 5) for I in range(8 ** k)) == 6039504


def test_lists_tile_every_leaf_exactly_once(orc):
    kap = 3
    nleaf = 8 ** kap
    for I in [0, 77, 300, 511, 146]:
        hits = np.zeros(nleaf, dtype=int)
        for J in orc.neighbours(kap, I):
            hits[J] += 1
        for k in range(2, kap + 1):
            A = I >> (3 * (kap - k))
            for J in orc.interaction_list(k, A):
                leaves = np.arange(J << (3 * (kap - k)), (J + 1) << (3 * (kap - k)))
                hits[leaves] += 1
        assert (hits == 1).all()


def test_interaction_offsets_are_the_316(orc):
    c = _coords(3)
    seen = set()
    for I in range(512):
        for J in orc.interaction_list(3, I):
            seen.add(tuple(c[J] - c[I]))
    assert len(seen) == 7 ** 3 - 3 ** 3


# --------------------------------------------------------------------------
# Training sets and EIM (Section 2, Algorithm 1)
# --------------------------------------------------------------------------
def test_training_sets_shape_and_domains(orc):
    for k, nx in [(2, 15 ** 3 - 5 ** 3), (3, 21 ** 3 - 5 ** 3)]:
        X, Y = orc.train_x(k), orc.train_y(k)
        l = 2.0 ** -(k + 1)
        assert len(X) == nx and len(Y) == 9 ** 3
        m = np.abs(X).max(1)
        assert (m >= 3 * l).all() and (m <= 1 - l + 1e-15).all()
        assert np.abs(Y).max() == l and (np.abs(Y) <= l).all()
        assert len(np.unique(X, axis=0)) == len(X)


def _K(z, kern):
    r2 = (z * z).sum(-1)
    return {"inv_r": lambda: 1 / np.sqrt(r2), "quad": lambda: r2, "one": lambda: np.ones_like(r2),
            "exp_r2": lambda: np.exp(-r2)}[kern]()


def _interp(e, x, y, kern, orc):
    """I_d K(x, y) = sum_{l,m} Delta_lm K(x, y_l) K(x_m, y), Eq. (approx2)."""
    kx = _K(x[:, None, :] - e["Y"][None], kern)              # K(x, y_l)
    ky = _K(e["X"][:, None, :] - y[None], kern)              # K(x_m, y)
    dk = np.stack([orc.apply_delta(e["Gamma"], e["B"], ky[:, j]) for j in range(ky.shape[1])], 1)
    return kx @ dk


@pytest.fixture(scope="module")
def eim3(orc):
    X, Y = orc.train_x(3), orc.train_y(3)
    return X, Y, orc.eim("inv_r", X, Y, 1e-6)


def test_eim_structure_and_factorisation(orc, eim3):
    X, Y, e = eim3
    d = e["d"]
    B, G = e["B"], e["Gamma"]
    assert 100 < d < 300
    np.testing.assert_array_equal(np.diag(B), np.ones(d))
    assert np.all(np.triu(B, 1) == 0) and np.all(np.triu(G, 1) == 0)
    assert np.abs(B).max() <= 1.0 + 1e-12            # |q_m| <= 1 by the argmax
    A = _K(e["X"][:, None] - e["Y"][None], "inv_r")    # A_kl = K(x_k, y_l)
    assert np.abs(G @ B.T - A).max() <= 1e-12 * np.abs(A).max()
    np.testing.assert_allclose(np.abs(np.diag(G)), e["piv"][:d], rtol=0)
    assert e["eps_est"] <= 1e-6 and e["piv"][d] / e["piv"][0] == e["eps_est"]


def test_eim_pivots_are_greedy_argmax(orc, eim3):
    """Each pivot maximises |delta_k K| over the grid, with delta_k K rebuilt
    from the four-summation form of the first k terms."""
    X, Y, e = eim3
    sub_x = np.concatenate([e["ia"], np.arange(0, len(X), 97)])
    Aall = _K(X[sub_x][:, None] - Y[None], "inv_r")
    for k in [1, 5, 40, e["d"] - 1]:
        ek = dict(X=e["X"][:k], Y=e["Y"][:k], Gamma=e["Gamma"][:k, :k], B=e["B"][:k, :k])
        R = Aall - _interp(ek, X[sub_x], Y, "inv_r", orc)
        a, b = e["ia"][k], e["ib"][k]
        ra = np.where(sub_x == a)[0][0]
        assert abs(abs(R[ra, b]) - e["piv"][k]) <= 1e-9 * e["piv"][0]
        assert np.abs(R).max() <= e["piv"][k] * (1 + 1e-7) + 1e-12 * e["piv"][0]


def test_eim_interpolation_property(orc, eim3):
    """Property 2.1: I_d K(x, y_m) = K(x, y_m) and I_d K(x_m, y) = K(x_m, y)."""
    X, Y, e = eim3
    l = 2.0 ** -4
    g = wl.rng(4)
    xr = g.uniform(-1 + l, 1 - l, size=(400, 3))
    xr = xr[np.abs(xr).max(1) >= 3 * l]
    yr = g.uniform(-l, l, size=(300, 3))
    a = _interp(e, xr, e["Y"], "inv_r", orc)
    ref = _K(xr[:, None] - e["Y"][None], "inv_r")
    assert np.abs(a - ref).max() <= 1e-10 * np.abs(ref).max()
    b = _interp(e, e["X"], yr, "inv_r", orc)
    ref = _K(e["X"][:, None] - yr[None], "inv_r")
    assert np.abs(b - ref).max() <= 1e-10 * np.abs(ref).max()
    # off the grid the error stays within a small factor of the estimate
    c = _interp(e, xr, yr, "inv_r", orc)
    ref = _K(xr[:, None] - yr[None], "inv_r")
    assert np.abs(c - ref).max() <= 50 * e["eps_est"] * e["piv"][0]


@pytest.mark.parametrize("kern,rank", [("quad", 5), ("one", 1)])
def test_eim_exact_on_low_rank_kernels(orc, kern, rank):
    X, Y = orc.train_x(2), orc.train_y(2)
    e = orc.eim(kern, X, Y, 1e-10)
    assert e["d"] == rank
    g = wl.rng(9)
    xr = g.uniform(-0.875, 0.875, size=(200, 3))
    yr = g.uniform(-0.125, 0.125, size=(200, 3))
    ref = _K(xr[:, None] - yr[None], kern)
    assert np.abs(_interp(e, xr, yr, kern, orc) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_eim_convergence_tracks_estimate(orc):
    """Section 2: the error estimate decreases with d and tracks the error."""
    X, Y = orc.train_x(2), orc.train_y(2)
    g = wl.rng(10)
    xr = g.uniform(-0.875, 0.875, size=(300, 3))
    xr = xr[np.abs(xr).max(1) >= 0.375]
    yr = g.uniform(-0.125, 0.125, size=(200, 3))
    ref = _K(xr[:, None] - yr[None], "inv_r")
    ds, errs, ests = [], [], []
    for eps in [1e-2, 1e-3, 1e-4, 1e-5, 1e-6]:
        e = orc.eim("inv_r", X, Y, eps)
        err = np.abs(_interp(e, xr, yr, "inv_r", orc) - ref).max() / np.abs(ref).max()
        ds.append(e["d"]); errs.append(err); ests.append(e["eps_est"])
        assert e["eps_est"] <= eps
        assert err <= 50 * e["eps_est"]
    assert ds == sorted(ds) and len(set(ds)) == len(ds)
    assert errs[-1] < errs[0] * 5e-3
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_apply_delta_is_inverse_of_A(orc, eim3):
    """Delta = B^-t Gamma^-1 = A^-1 (Section 2, reading of Gamma as lower)."""
    X, Y, e = eim3
    d = e["d"]
    A = _K(e["X"][:, None] - e["Y"][None], "inv_r")
    v = wl.rng(3).standard_normal(d)
    w = orc.apply_delta(e["Gamma"], e["B"], A @ v)     # Delta A v = v
    assert np.abs(w - v).max() <= 1e-6 * np.abs(v).max()
    u = orc.apply_delta(e["Gamma"], e["B"], v, transpose=True)   # A^t Delta^t v = v
    assert np.abs(A.T @ u - v).max() <= 1e-8 * np.abs(v).max() * np.abs(A).max() * d


# --------------------------------------------------------------------------
# O2: Algorithm 3 + near field
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern", ["quad", "one"])
@pytest.mark.parametrize("depth", [2, 3, 4])
def test_eifmm_exact_for_separable_kernels(orc, kern, depth):
    """With an exact rank-d kernel every step of Algorithm 3 is exact, so O2
    must equal the direct sum to rounding at every tree depth."""
    x = wl.uniform_cube(1500, 30 + depth)
    s = wl.sigma_uniform(1500, 2, 31)
    lv = orc.build_levels(kern, 1.0, depth, 1e-10)
    assert all(lv[k]["d"] == {"quad": 5, "one": 1}[kern] for k in lv)
    f2, dm = orc.eifmm(kern, 1.0, [0, 0, 0], depth, lv, x, x, s, dump=True)
    f1 = orc.direct_sum(kern, x, x, s)
    assert np.linalg.norm(f2 - f1) / np.linalg.norm(f1) <= 1e-12
    assert dm["domain_violations"] == 0
    # the far field alone is a large part of the answer for these kernels
    assert np.linalg.norm(dm["f_far"]) > 0.1 * np.linalg.norm(f1)


@pytest.fixture(scope="module")
def c1_levels(orc):
    return {eps: orc.build_levels("inv_r", 1.0, 3, eps) for eps in (1e-4, 1e-6)}


def test_eifmm_inv_r_c1(orc, c1_levels):
    x = wl.uniform_cube(4096, 1)
    s = wl.sigma_uniform(4096, 1, 101)
    f1 = orc.direct_sum("inv_r", x, x, s)
    errs = []
    for eps in (1e-4, 1e-6):
        f2, dm = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, c1_levels[eps], x, x, s, dump=True)
        err = np.linalg.norm(f2 - f1) / np.linalg.norm(f1)
        errs.append(err)
        assert err <= eps
        assert dm["domain_violations"] == 0
        assert dm["m2l_pairs"] == 3096 + 53352
        np.testing.assert_allclose(dm["f_far"] + dm["f_near"], f2, rtol=1e-14, atol=1e-14)
    assert errs[1] < errs[0] / 5


def test_eifmm_p2p_pairs_brute_force(orc, c1_levels):
    x = wl.uniform_cube(600, 8)
    s = wl.sigma_uniform(600, 1, 9)
    _, dm = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, c1_levels[1e-4], x, x, s, dump=True)
    c = np.minimum(np.floor(x * 8).astype(int), 7)
    near = (np.abs(c[:, None, :] - c[None]).max(-1) <= 1).sum() - len(x)
    assert dm["p2p_pairs"] == near


def test_eifmm_monolevel_is_algorithm2(orc):
    """Depth 2: only level 2 carries a far field, Algorithm 3 = Algorithm 2."""
    x = wl.uniform_cube(2000, 40)
    s = wl.sigma_uniform(2000, 1, 41)
    lv = orc.build_levels("inv_r", 1.0, 2, 1e-6)
    f2 = orc.eifmm("inv_r", 1.0, [0, 0, 0], 2, lv, x, x, s)
    f1 = orc.direct_sum("inv_r", x, x, s)
    assert np.linalg.norm(f2 - f1) / np.linalg.norm(f1) <= 1e-6


def test_eifmm_multi_rhs_and_separate_sets(orc, c1_levels):
    lv = c1_levels[1e-4]
    y = wl.gaussian_mixture(3000, 50)
    x = wl.uniform_cube(800, 51)
    s = wl.sigma_uniform(3000, 3, 52)
    f = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lv, x, y, s, exclude_self=False)
    for r in range(3):
        fr = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lv, x, y, s[:, r], exclude_self=False)
        np.testing.assert_array_equal(f[:, r], fr[:, 0])
    f1 = orc.direct_sum("inv_r", x, y, s, exclude_self=False)
    assert np.linalg.norm(f - f1) / np.linalg.norm(f1) <= 1e-4


def test_eifmm_translated_domain(orc):
    """Translation invariance (Section 3.1): shifting Omega and all points
    together leaves f unchanged."""
    x = wl.uniform_cube(1500, 60)
    s = wl.sigma_uniform(1500, 1, 61)
    lv = orc.build_levels("inv_r", 2.0, 3, 1e-5)
    lo = np.array([-3.0, 0.5, 7.0])
    fa = orc.eifmm("inv_r", 2.0, [0, 0, 0], 3, lv, 2 * x, 2 * x, s)
    fb = orc.eifmm("inv_r", 2.0, lo, 3, lv, lo + 2 * x, lo + 2 * x, s)
    assert np.linalg.norm(fa - fb) / np.linalg.norm(fa) <= 1e-9
    f1 = orc.direct_sum("inv_r", 2 * x, 2 * x, s)
    assert np.linalg.norm(fa - f1) / np.linalg.norm(f1) <= 1e-5


def test_eim_inhomogeneous_kernel_rank_decreases_with_depth(orc):
    """Section 5.4: for e^{-r^2} the EIM selects fewer points deeper in the
    tree (the approximation problem gets easier as boxes shrink)."""
    d = [orc.eim("exp_r2", orc.train_x(k), orc.train_y(k), 1e-6)["d"] for k in (2, 3, 4)]
    assert d[0] > d[1] > d[2]


def test_sphere_points_on_surface():
    x = wl.sphere_surface(1000, 3)
    r = np.linalg.norm(x - 0.5, axis=1)
    assert np.abs(r - 0.5).max() < 1e-12 and (x >= 0).all() and (x <= 1).all()


# --------------------------------------------------------------------------
# M2L compression, Section 4.2 (first stage), and the operator K^delta Delta
# --------------------------------------------------------------------------
def _filters_by_definition(s, eps):
    """The two filters written as the inequalities that define them: (i) j
    with s_j / s_0 <= eps <= s_{j-1} / s_0 (0-based: the first value at or
    below eps is s_j, so j values are kept); (ii) the j with
    sum_{i<=j} s_i >= (1 - eps) sum s >= sum_{i<=j-1} s_i (1-based)."""
    n = len(s)
    r1 = n
    for j in range(1, n):
        if s[j] / s[0] <= eps <= s[j - 1] / s[0]:
            r1 = j
            break
    tot = math.fsum(s)
    r2 = n
    for j in range(1, n + 1):
        if math.fsum(s[:j]) >= (1 - eps) * tot >= math.fsum(s[:j - 1]):
            r2 = j
            break
    return r1, r2


@pytest.mark.parametrize("spec", ["geometric", "plateau", "cliff"])
def test_sarcmp_filters_match_their_definition(orc, spec):
    if spec == "geometric":
        s, eps = 0.5 ** np.arange(40.0), 1e-3
    elif spec == "plateau":
        s, eps = np.r_[np.ones(10), 1e-9 * np.ones(5)], 1e-4
    else:
        s, eps = np.r_[1.0, 0.5, 0.25, 1e-5, 1e-6, 1e-7, 1e-8], 1e-4
    assert orc.sarcmp_rank(s, eps) == _filters_by_definition(list(s), eps)


@pytest.fixture(scope="module")
def lv3(orc):
    return orc.build_levels("inv_r", 1.0, 3, 1e-4)


def test_m2l_operators_mirror_symmetry(orc, lv3):
    """An even kernel gives K^{-delta} = (K^delta)^t: the symmetric case in
    which one basis U serves both sides of C^delta = U^t K^delta U."""
    Kd = orc.m2l_operators("inv_r", 1.0, 3, lv3[3])
    for t in orc.FAR_SLOTS:
        np.testing.assert_allclose(Kd[342 - t], Kd[t].T, rtol=1e-13, atol=0)
    assert len(orc.FAR_SLOTS) == 316
    assert not Kd[171].any()  # delta = 0 is a neighbour offset


def test_sarcmp_basis_truncation_error(orc, lv3):
    """Eckart-Young: projecting K_fat on the r kept left singular vectors
    leaves exactly the discarded singular values (Frobenius norm)."""
    b = orc.sarcmp_basis("inv_r", 1.0, 3, lv3[3], 1e-4)
    U, r, s = b["U"], b["r"], b["s"]
    Kd = orc.m2l_operators("inv_r", 1.0, 3, lv3[3])
    Kfat = np.hstack([Kd[t] for t in orc.FAR_SLOTS])
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-12)
    res = np.linalg.norm(Kfat - U @ (U.T @ Kfat)) ** 2
    assert abs(res - np.sum(s[r:] ** 2)) <= 1e-9 * np.sum(s ** 2)
    assert r == max(b["r_i"], b["r_ii"]) and 0 < r < lv3[3]["d"]


def test_sarcmp_full_rank_is_the_plain_m2l(orc, lv3):
    """With r = d the basis is orthogonal and U C^delta U^t = K^delta."""
    x = wl.uniform_cube(3000, 21)
    s = wl.sigma_uniform(3000, 1, 22)
    f0 = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lv3, x, x, s)
    lvc = {k: dict(e, U=orc.sarcmp_basis("inv_r", 1.0, k, e, 1e-4, r=e["d"])["U"]) for k, e in lv3.items()}
    f1 = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lvc, x, x, s)
    assert np.linalg.norm(f1 - f0) <= 1e-11 * np.linalg.norm(f0)


def test_sarcmp_meets_the_tolerance(orc, lv3):
    """The compressed method against the exact sum: within eps, and the
    truncation is visible (the result moves by more than rounding)."""
    x = wl.uniform_cube(4096, 1)
    s = wl.sigma_uniform(4096, 1, 101)
    f1 = orc.direct_sum("inv_r", x, x, s)
    f0 = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lv3, x, x, s)
    lvc = {k: dict(e, U=orc.sarcmp_basis("inv_r", 1.0, k, e, 1e-4)["U"]) for k, e in lv3.items()}
    fc = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lvc, x, x, s)
    assert np.linalg.norm(fc - f1) <= 1e-4 * np.linalg.norm(f1)
    assert np.linalg.norm(fc - f0) > 1e-9 * np.linalg.norm(f0)


def test_m2l_operator_with_delta_folded_in(orc, lv3):
    """Steps 3-4 as one operator: sum_J K^delta (Delta W^J) equals
    sum_J (K^delta Delta) W^J, with the rows of K^delta Delta obtained by
    applying Delta^t (the oracle's own solves) to the rows of K^delta.  The
    folded operator is also far less sensitive to rounding of its input:
    W and the operator rounded to FP32 move g by ~1e-7, while What rounded
    after FP32 solves would not (the ill-conditioned Delta amplifies)."""
    e = lv3[3]
    x = wl.uniform_cube(4096, 1)
    s = wl.sigma_uniform(4096, 1, 101)
    _, dm = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, lv3, x, x, s, dump=True)
    W = dm["W"][3][::8, 0, :]  # multipole coefficients of 64 leaves
    Kd = orc.m2l_operators("inv_r", 1.0, 3, e)
    Wh = np.array([orc.apply_delta(e["Gamma"], e["B"], w) for w in W])
    np.testing.assert_allclose(Wh, dm["What"][3][::8, 0, :], rtol=0, atol=0)
    for t in (orc.FAR_SLOTS[0], orc.FAR_SLOTS[200]):
        K = Kd[t]
        M = np.array([orc.apply_delta(e["Gamma"], e["B"], row, transpose=True) for row in K])
        g_ref = Wh @ K.T
        np.testing.assert_allclose(W @ M.T, g_ref, rtol=0, atol=1e-10 * np.abs(g_ref).max())
        g32 = (W.astype(np.float32) @ M.T.astype(np.float32)).astype(np.float64)
        assert np.linalg.norm(g32 - g_ref) <= 1e-6 * np.linalg.norm(g_ref)
