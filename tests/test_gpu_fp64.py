"""GPU parity of the tree, the EIM and the FP64 EIFMM against the CPU checker.

Tolerances:
  * integer work (Morton keys, permutation, leaf offsets, EIM pivots): exact;
  * EIM factors for kernels without transcendental functions: bit-exact (both
    sides evaluate the same IEEE operations without fused multiply-add);
  * FP64 evaluation: the two implementations differ only in summation order
    and contraction, i.e. relative rounding of a few 1e-16 per operation.
    The quantities that are well conditioned functions of the input (W, g, l,
    f_far, f_near, f) are compared at 1e-12 relative to their max-norm.  Wh
    = Delta W and lhat = Delta^t l go through solves with cond(A) up to
    ~1e9, so they are compared by their backward error (A Wh = W) at 1e-12
    and forward at 1e-6.
"""
import numpy as np
import pytest

from paper_1408_0210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_0210_gb300 import build, eifmm
    build.build()
    eifmm.lib()
    return eifmm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------------------
# tree: bit-exact
# --------------------------------------------------------------------------
TREE_CASES = [
    ("uniform", 4096, 3),
    ("uniform", 2049, 2),       # one full radix tile plus a ragged tail of 1
    ("uniform", 1, 4),
    ("gauss", 20000, 5),
    ("uniform", 1 << 20, 5),    # the 1M-point workload
    ("gauss", 300000, 7),       # 21-bit keys, 3 radix passes
]


@pytest.mark.parametrize("kind,n,depth", TREE_CASES)
def test_tree_bit_exact(E, orc, kind, n, depth):
    x = wl.uniform_cube(n, 100 + n % 97) if kind == "uniform" else wl.gaussian_mixture(n, 3)
    if n > 8:
        x[0] = [1.0, 1.0, 0.0]
        x[1] = [0.5, 0.25, 0.75]
    t = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    keys, perm, off = t.export(0)
    ok, out = orc.morton_keys(x, [0, 0, 0], 1.0, depth)
    assert out == 0
    operm, ooff = orc.sort_leaves(ok, depth)
    np.testing.assert_array_equal(perm, operm)
    np.testing.assert_array_equal(keys, ok[operm])
    np.testing.assert_array_equal(off, ooff)


def test_tree_general_cube_and_separate_targets(E, orc):
    lo = np.array([-2.0, 0.5, 3.0])
    L = 4.0
    src = lo + L * wl.uniform_cube(5000, 1)
    tgt = lo + L * wl.gaussian_mixture(3000, 2)
    t = E.eifmm_tree_build(dev(src), dev(tgt), lo, L, 4, False)
    for which, pts in ((0, src), (1, tgt)):
        keys, perm, off = t.export(which)
        ok, _ = orc.morton_keys(pts, lo, L, 4)
        operm, ooff = orc.sort_leaves(ok, 4)
        np.testing.assert_array_equal(perm, operm)
        np.testing.assert_array_equal(off, ooff)


def test_tree_rejects_points_outside(E):
    x = wl.uniform_cube(100, 5)
    x[7, 1] = 1.0 + 1e-12
    with pytest.raises(E.EifmmError, match="outside"):
        E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, 3, True)


# --------------------------------------------------------------------------
# EIM (Algorithm 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kern,level,eps", [("inv_r", 2, 1e-6), ("inv_r", 3, 1e-4),
                                            ("quad", 3, 1e-10), ("one", 2, 1e-10),
                                            ("inv_r", 5, 1e-5)])
def test_eim_bit_exact(E, orc, kern, level, eps):
    X, Y = orc.train_x(level), orc.train_y(level)
    g = E.eifmm_eim_build(kern, X, Y, eps)
    o = orc.eim(kern, X, Y, eps)
    assert g["d"] == o["d"]
    np.testing.assert_array_equal(g["ia"], o["ia"])
    np.testing.assert_array_equal(g["ib"], o["ib"])
    np.testing.assert_array_equal(g["Gamma"], o["Gamma"])
    np.testing.assert_array_equal(g["B"], o["B"])
    np.testing.assert_array_equal(g["piv"], o["piv"])
    assert g["eps_est"] == o["eps_est"]


def test_eim_transcendental_kernel_valid(E, orc):
    """exp() differs between libm and CUDA in the last bit, so pivots may be
    chosen differently among near-ties; what is unique is checked: the
    factorisation A = Gamma B^t at the chosen points and the estimate."""
    X, Y = orc.train_x(3), orc.train_y(3)
    g = E.eifmm_eim_build("config3", X, Y, 1e-6)
    o = orc.eim("config3", X, Y, 1e-6)
    assert abs(g["d"] - o["d"]) <= 3
    z = g["X"][:, None, :] - g["Y"][None]
    A = np.array([[orc.kernel("config3", zz) for zz in row] for row in z[:40, :40]])
    GBt = (g["Gamma"] @ g["B"].T)[:40, :40]
    assert np.abs(GBt - A).max() <= 1e-12 * np.abs(A).max()
    assert g["eps_est"] <= 1e-6


# --------------------------------------------------------------------------
# FP64 evaluation vs the CPU EIFMM
# --------------------------------------------------------------------------
def _levels(orc, kern, depth, eps):
    return orc.build_levels(kern, 1.0, depth, eps)


def _solve_residual(Wh, W, lv):
    """max |A Wh - W| / max |W| with A_kl = K(x_k, y_l) = 1/|x_k - y_l|."""
    A = 1.0 / np.linalg.norm(lv["X"][:, None] - lv["Y"][None], axis=-1)
    return float(np.abs(np.einsum("kl,brl->brk", A, Wh) - W).max() / np.abs(W).max())


@pytest.fixture(scope="module")
def c1(E, orc):
    """The 4096-point, depth-3, eps = 1e-6 workload (targets = sources)."""
    n, depth, eps = 4096, 3, 1e-6
    x = wl.uniform_cube(n, 1)
    s = wl.sigma_uniform(n, 1, 101)
    lv = _levels(orc, "inv_r", depth, eps)
    f2, dm = orc.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv, x, x, s, dump=True)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), f, "fp64")
    torch.cuda.synchronize()
    return dict(x=x, s=s, lv=lv, f2=f2, dm=dm, ops=ops, tree=tree, f=f.cpu().numpy(), depth=depth)


def test_fp64_c1_result(E, orc, c1):
    f = c1["f"]
    assert rel2(f, c1["f2"][:, 0]) <= 1e-12
    assert relmax(f, c1["f2"][:, 0]) <= 1e-12
    f1 = orc.direct_sum("inv_r", c1["x"], c1["x"], c1["s"])[:, 0]
    assert rel2(f, f1) <= 1e-6


def test_fp64_c1_every_step(E, c1):
    t, dm, lv, depth = c1["tree"], c1["dm"], c1["lv"], c1["depth"]
    for k in range(2, depth + 1):
        d = lv[k]["d"]
        W = E.eifmm_debug_export(t, 0, k, d)
        assert relmax(W, dm["W"][k]) <= 1e-12, f"W level {k}"
        Wh = E.eifmm_debug_export(t, 1, k, d)
        assert _solve_residual(Wh, dm["W"][k], lv[k]) <= 1e-12, f"Wh backward level {k}"
        assert relmax(Wh, dm["What"][k]) <= 1e-6, f"Wh forward level {k}"
        g = E.eifmm_debug_export(t, 2, k, d)
        assert relmax(g, dm["g"][k]) <= 1e-12, f"g level {k}"
        lk = E.eifmm_debug_export(t, 3, k, d)
        assert relmax(lk, dm["l"][k]) <= 1e-12, f"l level {k}"
    lh = E.eifmm_debug_export(t, 4, depth, lv[depth]["d"])
    assert relmax(lh, dm["lhat"]) <= 1e-6
    ffar = E.eifmm_debug_export(t, 5, depth, 0)
    fnear = E.eifmm_debug_export(t, 6, depth, 0)
    assert relmax(ffar, dm["f_far"]) <= 1e-12
    assert relmax(fnear, dm["f_near"]) <= 1e-13


@pytest.mark.parametrize("kern,depth", [("quad", 2), ("quad", 4), ("one", 3)])
def test_fp64_exact_for_separable_kernels(E, orc, kern, depth):
    x = wl.uniform_cube(3000, 70 + depth)
    s = wl.sigma_uniform(3000, 1, 71)
    ops = E.eifmm_ops_build(kern, 1.0, depth, 1e-10)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    f = torch.zeros(3000, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), f, "fp64")
    f1 = orc.direct_sum(kern, x, x, s)[:, 0]
    assert rel2(f.cpu().numpy(), f1) <= 1e-12


def test_fp64_multi_rhs_separate_sets_nonuniform(E, orc):
    depth, eps = 4, 1e-5
    src = wl.gaussian_mixture(6000, 11)
    tgt = wl.uniform_cube(2500, 12)
    s = wl.sigma_uniform(6000, 3, 13)
    lv = _levels(orc, "inv_r", depth, eps)
    f2 = orc.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv, tgt, src, s, exclude_self=False)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    tree = E.eifmm_tree_build(dev(src), dev(tgt), (0, 0, 0), 1.0, depth, False)
    sd = torch.from_numpy(np.asfortranarray(s)).to("cuda").T.contiguous().T
    f = torch.zeros(3, 2500, dtype=torch.float64, device="cuda").T
    E.eifmm_evaluate(tree, ops, sd, f, "fp64")
    assert relmax(f.cpu().numpy(), f2) <= 1e-12


def test_fp64_host_entry_and_batched(E, orc, c1):
    fh = E.eifmm_evaluate_host(c1["tree"], c1["ops"], c1["s"])
    assert relmax(fh[:, 0], c1["f"]) == 0.0
    xs = [wl.uniform_cube(n, 200 + n) for n in (700, 1500)]
    ss = [wl.sigma_uniform(len(x), 1, 300 + len(x))[:, 0] for x in xs]
    trees = [E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, 3, True) for x in xs]
    fs = [torch.zeros(len(x), dtype=torch.float64, device="cuda") for x in xs]
    E.eifmm_evaluate_batched(trees, [dev(s) for s in ss], fs, c1["ops"], "fp64")
    for x, s, f in zip(xs, ss, fs):
        f2 = orc.eifmm("inv_r", 1.0, [0, 0, 0], 3, c1["lv"], x, x, s)[:, 0]
        assert relmax(f.cpu().numpy(), f2) <= 1e-12


def test_fp64_degenerate_inputs(E, orc):
    ops = E.eifmm_ops_build("inv_r", 1.0, 2, 1e-4)
    # all points in one leaf: only the near field
    x = 0.01 * wl.uniform_cube(50, 1)
    s = wl.sigma_uniform(50, 1, 2)[:, 0]
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, 2, True)
    f = torch.zeros(50, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s), f, "fp64")
    np.testing.assert_allclose(f.cpu().numpy(), orc.direct_sum("inv_r", x, x, s)[:, 0], rtol=1e-13)
    # a single point: f = 0
    x1 = np.array([[0.3, 0.6, 0.9]])
    t1 = E.eifmm_tree_build(dev(x1), None, (0, 0, 0), 1.0, 2, True)
    f1 = torch.ones(1, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(t1, ops, dev(np.array([2.0])), f1, "fp64")
    assert f1.item() == 0.0
    # two far-apart points: the far field alone carries the interaction
    x2 = np.array([[0.05, 0.05, 0.05], [0.95, 0.95, 0.95]])
    t2 = E.eifmm_tree_build(dev(x2), None, (0, 0, 0), 1.0, 2, True)
    f2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(t2, ops, dev(np.array([1.0, -2.0])), f2, "fp64")
    ref = orc.direct_sum("inv_r", x2, x2, np.array([1.0, -2.0]))[:, 0]
    assert rel2(f2.cpu().numpy(), ref) <= 1e-4
    # depth / L mismatch between tree and operators
    t3 = E.eifmm_tree_build(dev(x2), None, (0, 0, 0), 1.0, 3, True)
    with pytest.raises(E.EifmmError, match="depth"):
        E.eifmm_evaluate(t3, ops, dev(np.array([1.0, -2.0])), f2, "fp64")


def test_direct_sum_matches_checker(E, orc):
    x = wl.uniform_cube(5000, 90)
    y = wl.gaussian_mixture(7000, 91)
    s = wl.sigma_uniform(7000, 2, 92)
    idx = wl.sample_targets(5000, 300, 93)
    sd = torch.from_numpy(np.asfortranarray(s)).to("cuda").T.contiguous().T
    fg = E.eifmm_direct_sum("inv_r", dev(x), dev(y), sd, False, dev(idx)).cpu().numpy()
    fo = orc.direct_sum("inv_r", x, y, s, exclude_self=False, tgt_idx=idx)
    assert relmax(fg, fo) <= 1e-13
    fg = E.eifmm_direct_sum("config3", dev(x), dev(x), dev(s[:5000, 0]), True).cpu().numpy()
    fo = orc.direct_sum("config3", x, x, s[:5000, :1])
    assert relmax(fg, fo) <= 1e-12
