"""The benchmark configurations at full size, on the GPU, against the CPU
checker's exact sum (Eq. (1)) on sampled targets.

  C3   1,048,576 points from 8 Gaussians (std 0.05, centres U[0.2,0.8]^3,
       clipped), K = exp(-r)/r + 1/sqrt(r1^2 + 0.01 r2^2 + r3^2 + 1e-3),
       depth 5, per-level d from the estimate at eps = 1e-6, mixed and FP64
  C4a  262,144 uniform points, 1/r, depth 5, 64 sigma vectors, eps = 1e-6
  C4b  32 problems of log-uniform size in [16384, 262144], own points and
       trees (depth clamp(ceil(log8(N / 32)), 3, 5)), one operator set, one
       graph-captured batched launch, eps = 1e-6
  C5   16,777,216 uniform points, 1/r, depth 7, 8 sigma vectors N(0, 1),
       mixed at eps = 1e-5

Tolerances: the configured eps for the 1/r configurations (rel-L2 over the
sampled targets, the worst right-hand side).  C3's kernel is anisotropic: boxes
separated only along y are not well separated for it, and the method itself
stays far from the exact sum there (measured 8.8e-2 on this workload, with the
FP64 path), so C3 checks the mixed path against the FP64 one to eps and both
against the exact sum to 0.15.
"""
import math

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


def devcols(s):
    """(n, R) host array -> column-major CUDA tensor (n, R)."""
    return torch.from_numpy(np.asfortranarray(s)).to("cuda").T.contiguous().T


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c3_gaussian_mixture_config3_kernel(E, orc):
    n, depth, eps = 1 << 20, 5, 1e-6
    x = wl.gaussian_mixture(n, 3)
    s = wl.sigma_uniform(n, 1, 103)
    ops = E.eifmm_ops_build("config3", 1.0, depth, eps)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    _, _, off = tree.export(1)
    cnt = np.diff(off)
    assert cnt.max() > 32 * 20 and (cnt == 0).sum() > 0  # hot and empty leaves
    f = {}
    for prec in ("fp64", "mixed"):
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        E.eifmm_evaluate(tree, ops, dev(s[:, 0]), out, prec)
        f[prec] = out.cpu().numpy()
        assert np.isfinite(f[prec]).all()
    assert rel2(f["mixed"], f["fp64"]) <= eps
    idx = wl.sample_targets(n, 256, 33)
    f1 = orc.direct_sum("config3", x, x, s, tgt_idx=idx)[:, 0]
    for prec in ("fp64", "mixed"):
        assert rel2(f[prec][idx], f1) <= 0.15, prec


def test_measured_rates_are_sane(E):
    r = E.eifmm_measure_rates()
    assert r["ffma_per_s"] > r["rsqrt_per_s"] > 0
    assert r["ffma_per_s"] > r["dfma_per_s"] > 0


def test_c4a_many_rhs_full_size(E, orc):
    n, depth, eps, R = 262144, 5, 1e-6, 64
    x = wl.uniform_cube(n, 4)
    s = wl.sigma_uniform(n, R, 104)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    sd = devcols(s)
    f = {}
    for prec in ("fp64", "mixed"):
        out = torch.zeros(R, n, dtype=torch.float64, device="cuda").T
        E.eifmm_evaluate(tree, ops, sd, out, prec)
        f[prec] = out.cpu().numpy()
    assert max(rel2(f["mixed"][:, r], f["fp64"][:, r]) for r in range(R)) <= eps / 2
    idx = wl.sample_targets(n, 192, 44)
    f1 = orc.direct_sum("inv_r", x, x, s, tgt_idx=idx)
    for prec in ("fp64", "mixed"):
        assert max(rel2(f[prec][idx, r], f1[:, r]) for r in range(R)) <= eps, prec


def test_c4b_uneven_batch_one_graph_launch(E, orc):
    eps = 1e-6
    sizes = wl.batch_sizes(32, 16384, 262144, 40)
    depths = [min(5, max(3, math.ceil(math.log(nn / 32, 8)))) for nn in sizes]
    ops = E.eifmm_ops_build("inv_r", 1.0, max(depths), eps)
    xs = [wl.uniform_cube(nn, 40 + p) for p, nn in enumerate(sizes)]
    ss = [wl.sigma_uniform(nn, 1, 140 + p) for p, nn in enumerate(sizes)]
    trees = [E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, d, True) for x, d in zip(xs, depths)]
    sd = [dev(s[:, 0]) for s in ss]
    fb = [torch.zeros(nn, dtype=torch.float64, device="cuda") for nn in sizes]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        E.eifmm_evaluate_batched(trees, sd, fb, ops, "mixed", stream)   # direct pass + capture
        for f in fb:
            f.zero_()
        n0 = E.eifmm_kernel_launches()
        E.eifmm_evaluate_batched(trees, sd, fb, ops, "mixed", stream)   # one graph launch
        assert E.eifmm_kernel_launches() == n0
    stream.synchronize()
    for p in range(len(sizes)):
        fi = torch.zeros(sizes[p], dtype=torch.float64, device="cuda")
        E.eifmm_evaluate(trees[p], ops, sd[p], fi, "mixed")
        assert torch.equal(fi, fb[p]), p
    for p in (0, 7, 19, 31):
        idx = wl.sample_targets(sizes[p], 256, 200 + p)
        f1 = orc.direct_sum("inv_r", xs[p], xs[p], ss[p], tgt_idx=idx)[:, 0]
        assert rel2(fb[p].cpu().numpy()[idx], f1) <= eps, (p, sizes[p], depths[p])


def test_c5_sixteen_million_points_depth7(E, orc):
    n, depth, eps, R = 1 << 24, 7, 1e-5, 8
    x = wl.uniform_cube(n, 5)
    s = wl.sigma_normal(n, R, 105)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    out = torch.zeros(R, n, dtype=torch.float64, device="cuda").T
    E.eifmm_evaluate(tree, ops, devcols(s), out, "mixed")
    idx = wl.sample_targets(n, 96, 55)
    fg = out[torch.from_numpy(idx).to("cuda")].cpu().numpy()
    del out, tree
    torch.cuda.empty_cache()
    f1 = orc.direct_sum("inv_r", x, x, s, tgt_idx=idx)
    assert np.isfinite(fg).all()
    assert max(rel2(fg[:, r], f1[:, r]) for r in range(R)) <= eps
