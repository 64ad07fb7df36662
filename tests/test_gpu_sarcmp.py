"""The M2L compression of Section 4.2 (first stage) on the GPU, FP64 far
field, against the CPU checker's compressed method (O2 with the basis U).

* Ranks: the counts of the two filters and the kept rank equal the
  checker's (its truncated SVD of K_fat); the singular values come from the
  eigenvalues of K_fat K_fat^t on the GPU side.
* Basis: the GPU's U spans the checker's subspace up to what the truncation
  itself drops: || (U U^t - U_o U_o^t) K_fat ||_F <= eps s_0 (s_0 the largest
  singular value).  Both keep every direction above eps s_0; they may differ
  by a rotation among directions whose singular values lie near the cut,
  which the squared singular values of the Gram matrix do not resolve
  below about 1e-8 s_0.
* Method: the FP64 path with the GPU's U against O2 run with the same U,
  1e-12 of the largest |f| (only the summation order differs); both within
  eps of the exact sum.  Tier 3 runs the compressed M2L in FP32 pairs: its g
  at every level agrees with the FP64 compressed M2L to 1e-10 of the largest
  entry (about 48 bits per pair, the tier-3 criterion of the uncompressed
  M2L), and its f stays within eps of the exact sum.
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


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_compressed_fp64_path_matches_checker(E, orc, eps):
    n, depth = 4096, 3
    x = wl.uniform_cube(n, 1)
    s = wl.sigma_uniform(n, 1, 101)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    ranks = ops.compress(eps)
    lv = orc.build_levels("inv_r", 1.0, depth, eps)
    for k in range(2, depth + 1):
        b = ops.basis(k)
        ob = orc.sarcmp_basis("inv_r", 1.0, k, lv[k], eps)
        assert (b["r_i"], b["r_ii"], b["r"]) == (ob["r_i"], ob["r_ii"], ob["r"]), k
        assert ranks[k] == ob["r"] and b["r"] < b["d"]
        Kd = orc.m2l_operators("inv_r", 1.0, k, lv[k])
        Kfat = np.hstack([Kd[t] for t in orc.FAR_SLOTS])
        P, Po = b["U"] @ b["U"].T, ob["U"] @ ob["U"].T
        assert np.linalg.norm((P - Po) @ Kfat) <= eps * ob["s"][0], k
        lv[k] = dict(lv[k], U=b["U"])
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), f, "fp64")
    torch.cuda.synchronize()
    fg = f.cpu().numpy()
    f2 = orc.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv, x, x, s)[:, 0]
    assert np.abs(fg - f2).max() <= 1e-12 * np.abs(f2).max()
    f1 = orc.direct_sum("inv_r", x, x, s)[:, 0]
    assert rel2(fg, f1) <= eps
    g64 = {k: E.eifmm_debug_export(tree, 2, k, lv[k]["d"]) for k in range(2, depth + 1)}
    # tier 3: the compressed M2L in FP32 pairs
    ops.plan(3)
    fm = torch.zeros(n, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), fm, "mixed")
    torch.cuda.synchronize()
    for k in range(2, depth + 1):
        gk = E.eifmm_debug_export(tree, 2, k, lv[k]["d"])
        assert np.abs(gk - g64[k]).max() <= 1e-10 * np.abs(g64[k]).max(), k
    assert rel2(fm.cpu().numpy(), f1) <= eps
    # eps = 0 removes the compression: the plain FP64 path again
    assert all(r == 0 for r in ops.compress(0.0).values())
    f0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), f0, "fp64")
    lv0 = orc.build_levels("inv_r", 1.0, depth, eps)
    f20 = orc.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv0, x, x, s)[:, 0]
    assert np.abs(f0.cpu().numpy() - f20).max() <= 1e-12 * np.abs(f20).max()


def test_compressed_tier3_full_size(E, orc):
    """1,048,576 points, depth 5, eps = 1e-6: tier 3 with the compressed M2L
    stays within eps of the exact sum on sampled targets."""
    n, depth, eps = 1 << 20, 5, 1e-6
    x = wl.uniform_cube(n, 2)
    s = wl.sigma_uniform(n, 1, 102)
    ops = E.eifmm_ops_build("inv_r", 1.0, depth, eps)
    assert ops.plan() == 3
    ranks = ops.compress(eps)
    assert all(0 < ranks[k] < ops.error_estimate(k)[1] for k in range(2, depth + 1))
    tree = E.eifmm_tree_build(dev(x), None, (0, 0, 0), 1.0, depth, True)
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    E.eifmm_evaluate(tree, ops, dev(s[:, 0]), f, "mixed")
    idx = wl.sample_targets(n, 400, 55)
    f1 = orc.direct_sum("inv_r", x, x, s, tgt_idx=idx)[:, 0]
    assert rel2(f.cpu().numpy()[idx], f1) <= eps
