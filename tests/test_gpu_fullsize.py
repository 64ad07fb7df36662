"""The 1,048,576-point, depth-5 workload (K = 1/r, eps = 1e-4) element by
element: the FP64 path and the tensor-core tier 0 against the CPU EIFMM (O2)
at every target, and the level-5 M2L of the transposed tcgen05 kernel
against an FP64 M2L on chosen target boxes (corners, edges, faces, inside).

Per-target bound of tier 0 (derived from its arithmetic):
  |f_i - f2_i| <= tau_far * F + tau_near * N_i
  F   = max_i |f_far,i| of O2: the far field's errors are relative to the
        size of the multipole and local expansions, not to f_i itself.  The
        BF16 hi+lo planes keep about 16 bits per product of the M2L (2^-16 =
        1.5e-5 per term), and the FP32 P2M, M2M, L2L, Delta^t and L2P steps
        add about 1e-6; tau_far = 2e-5.
  N_i = sum over the near field of |sigma_j| k(x_i - y_j) (O2's near field
        with |sigma|): every near term carries the relative error of
        rsqrt.approx (2^-22.9), one FP32 product and a share of at most 128
        FP32 additions before a compensated flush (127 * 2^-24 = 7.6e-6), plus
        the rounding of the leaf-local FP32 coordinates (about 5e-9 absolute,
        i.e. 5e-9 / r relative; 5e-5 at the closest pairs of 2^20 uniform
        points, r ~ 1e-4); tau_near = 1e-4.
"""
import numpy as np
import pytest

from paper_1408_0210_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, DEPTH, EPS = 1 << 20, 5, 1e-4
TAU_FAR, TAU_NEAR = 2e-5, 1e-4


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


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def big(E, orc):
    x = wl.uniform_cube(N, 2)
    s = wl.sigma_uniform(N, 1, 102)
    lv = orc.build_levels("inv_r", 1.0, DEPTH, EPS)
    f2, dm = orc.eifmm("inv_r", 1.0, [0, 0, 0], DEPTH, lv, x, x, s, dump=True)
    # the near field with |sigma|: the size N_i of every target's near sum
    _, dabs = orc.eifmm("inv_r", 1.0, [0, 0, 0], DEPTH, lv, x, x, np.abs(s), dump=True)
    ops = E.eifmm_ops_build("inv_r", 1.0, DEPTH, EPS)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, DEPTH, True)
    return dict(x=x, s=s, lv=lv, f2=f2[:, 0], ffar=dm["f_far"][:, 0], nabs=dabs["f_near"][:, 0],
                ops=ops, tree=tree)


def _eval(E, big, prec):
    f = torch.zeros(N, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(big["tree"], big["ops"], dev(big["s"][:, 0]), f, prec)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def test_fp64_full_size_every_target(E, orc, big):
    """FP64 path against O2 at all 2^20 targets (only the summation order
    differs), and against the exact sum on sampled targets."""
    fg = _eval(E, big, "fp64")
    assert relmax(fg, big["f2"]) <= 1e-12
    idx = wl.sample_targets(N, 400, 55)
    f1 = orc.direct_sum("inv_r", big["x"], big["x"], big["s"], tgt_idx=idx)[:, 0]
    assert rel2(fg[idx], f1) <= EPS


def test_tier0_full_size_every_target(E, big):
    """Tier 0 (BF16 hi+lo tcgen05 M2L, FP32 elsewhere) against O2 at every
    target within the per-target bound of the module docstring; the worst
    target and its leaf are reported."""
    assert big["ops"].plan(0) == 0
    fg = _eval(E, big, "mixed")
    F = np.abs(big["ffar"]).max()
    err = np.abs(fg - big["f2"])
    bound = TAU_FAR * F + TAU_NEAR * big["nabs"]
    ratio = err / bound
    w = int(np.argmax(ratio))
    leaf = tuple((np.minimum(big["x"][w] * 32, 31)).astype(int))
    print(f"tier 0: worst target {w} in leaf {leaf}: |err| {err[w]:.3e}, bound {bound[w]:.3e} "
          f"(ratio {ratio[w]:.3f}); rel-L2 vs O2 {rel2(fg, big['f2']):.3e}")
    assert ratio.max() <= 1.0
    assert rel2(fg, big["f2"]) <= 2e-5


def _coords(k, boxes):
    c = np.zeros((len(boxes), 3), dtype=np.int64)
    for i, key in enumerate(boxes):
        for b in range(k):
            for a in range(3):
                c[i, a] |= ((int(key) >> (3 * b + a)) & 1) << b
    return c


def _morton(k, c):
    key = 0
    for b in range(k):
        for a in range(3):
            key |= ((int(c[a]) >> b) & 1) << (3 * b + a)
    return key


def test_m2l_t256_level5_chosen_boxes(E, orc, big):
    """The leaf-level M2L of tier 0 (k_m2l_t256: every parity class of level 5
    has 4096 boxes, several 256-row tiles) against g^I = sum_J K^delta What^J
    (Eq. M2Lstep) in FP64 from the exported What, on the 8 corners, edge and
    face boxes and random inside boxes of all 8 parity classes."""
    assert big["ops"].plan(0) == 0
    _eval(E, big, "mixed")
    k = DEPTH
    n = 1 << k
    lv = big["lv"][k]
    d = lv["d"]
    Wh = E.eifmm_debug_export(big["tree"], 1, k, d)[:, 0]
    g = E.eifmm_debug_export(big["tree"], 2, k, d)[:, 0]
    rng = np.random.default_rng(7)
    pick = set()
    for cx in (0, 1, n - 2, n - 1):
        for cy in (0, 1, n - 2, n - 1):
            for cz in (0, 1, n - 2, n - 1):
                pick.add(_morton(k, (cx, cy, cz)))           # corners and near-corners
    for _ in range(120):
        c = rng.integers(0, n, 3)
        c[rng.integers(0, 3)] = rng.choice([0, n - 1])   # a face
        pick.add(_morton(k, c))
    for _ in range(120):
        pick.add(_morton(k, rng.integers(2, n - 2, 3)))  # inside
    boxes = np.array(sorted(pick))
    assert len(set(int(b) % 8 for b in boxes)) == 8
    Y = lv["Y"]
    l2 = 2.0 * 2.0 ** -(k + 1)
    cI = _coords(k, boxes)
    gref = np.zeros((len(boxes), d))
    for i, I in enumerate(boxes):
        J = orc.interaction_list(k, int(I))
        dl = (_coords(k, J) - cI[i]) * l2                   # c_J - c_I
        for j, Jb in enumerate(J):
            Kd = 1.0 / np.linalg.norm(Y[:, None] - (Y[None] + dl[j]), axis=-1)
            gref[i] += Kd @ Wh[Jb]
    gb = g[boxes]
    e = np.abs(gb - gref).max(1) / np.abs(gref).max()
    print(f"level-5 M2L on {len(boxes)} boxes: worst box {int(boxes[np.argmax(e)])} "
          f"max-norm error {e.max():.3e} of max |g|")
    # BF16 hi+lo planes of K^delta Delta (~2^-17 relative) and FP32 sums
    assert e.max() <= 2e-5
