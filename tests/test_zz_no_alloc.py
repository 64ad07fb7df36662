"""The allocation-free bin/sort (eifmm_tree_sort_static) against the regular
tree build.

Some callers cannot allocate device memory (their memory is owned by another
allocator, or fixed in a budget when they start, or their loops cannot pay
for cudaMalloc's device-wide synchronisation); this entry point sorts into
caller-owned arrays with a static scratch array of the library.  Two calls in a row must reproduce the
regular entry point bit for bit (integer work), and the second call must not
see anything left over by the first.  The file is named to be collected last.
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


def test_static_sort_matches_tree_build_on_two_calls(E):
    cases = [(wl.gaussian_mixture(300000, 3), 7), (wl.uniform_cube(1 << 20, 2), 5)]
    for x, depth in cases:
        x[0] = [1.0, 1.0, 0.0]
        xd = torch.from_numpy(x).cuda()
        t = E.eifmm_tree_build(xd, None, (0, 0, 0), 1.0, depth, True)
        keys, perm, off = t.export(0)
        ks, ps, os_ = E.eifmm_tree_sort_static(xd, (0, 0, 0), 1.0, depth)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ks.cpu().numpy().view(np.uint32), keys)
        np.testing.assert_array_equal(ps.cpu().numpy(), perm)
        np.testing.assert_array_equal(os_.cpu().numpy().astype(np.int64), off)


def test_static_sort_limits_and_errors(E):
    too_many = torch.zeros((E.STATIC_SORT_MAX_POINTS + 1, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EifmmError, match="static scratch limit"):
        E.eifmm_tree_sort_static(too_many, (0, 0, 0), 1.0, 3)
    x = wl.uniform_cube(1000, 4)
    x[5, 2] = 1.5
    with pytest.raises(E.EifmmError, match="outside"):
        E.eifmm_tree_sort_static(torch.from_numpy(x).cuda(), (0, 0, 0), 1.0, 3)
    # a clean call after a failed one: the error counter starts at zero again
    ok = wl.uniform_cube(1000, 4)
    ks, ps, os_ = E.eifmm_tree_sort_static(torch.from_numpy(ok).cuda(), (0, 0, 0), 1.0, 3)
    assert int(os_[-1].item()) == 1000
