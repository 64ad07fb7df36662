"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/eifmm.h, validates arguments before touching the device,
and its host-side training sets equal the CPU checker's bit for bit."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_1408_0210_gb300 import build, eifmm
    build.build()
    eifmm.lib()
    return eifmm


def _declared():
    txt = open(os.path.join(ROOT, "include", "eifmm.h")).read()
    return sorted(set(re.findall(r"\b(eifmm_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_exports(E):
    names = _declared()
    assert len(names) >= 15
    lib = C.CDLL(E.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(E.EXPORTS) == names


def test_version_and_error_string(E):
    assert "sm_103a" in E.eifmm_version()
    assert isinstance(E.lib().eifmm_last_error(), bytes)


@pytest.mark.parametrize("level", [2, 3, 4, 5, 6, 7])
def test_training_sets_equal_checker(E, orc, level):
    X, Y = E.eifmm_training_sets(level)
    np.testing.assert_array_equal(X, orc.train_x(level))
    np.testing.assert_array_equal(Y, orc.train_y(level))
    X2, _ = E.eifmm_training_sets(level, L=3.0)
    np.testing.assert_array_equal(X2, orc.train_x(level, 3.0))


def test_argument_validation_without_device(E):
    L = E.lib()
    nx, ny = C.c_int64(), C.c_int64()
    assert L.eifmm_training_sets(1, 1.0, 9, None, C.byref(nx), None, C.byref(ny)) == 1
    assert L.eifmm_training_sets(3, -1.0, 9, None, C.byref(nx), None, C.byref(ny)) == 1
    assert L.eifmm_training_sets(3, 1.0, 1, None, C.byref(nx), None, C.byref(ny)) == 1
    h = C.c_void_p()
    lo = np.zeros(3)
    assert L.eifmm_tree_build(None, 10, None, 10, lo.ctypes.data, 1.0, 3, 0, None, C.byref(h)) == 1
    assert L.eifmm_tree_build(1, 10, 1, 10, lo.ctypes.data, 1.0, 1, 0, None, C.byref(h)) == 1
    assert L.eifmm_tree_build(1, 10, 1, 10, lo.ctypes.data, 1.0, 11, 0, None, C.byref(h)) == 1
    assert L.eifmm_tree_build(1, 10, 2, 10, lo.ctypes.data, 1.0, 3, 1, None, C.byref(h)) == 1
    assert b"exclude_self" in L.eifmm_last_error()
    X = np.zeros((4, 3)); Y = np.ones((4, 3))
    d = C.c_int(); est = C.c_double()
    buf = np.zeros(64)
    assert L.eifmm_eim_build(0, X.ctypes.data, 4, Y.ctypes.data, 4, 0.0, 4, C.byref(d), buf.ctypes.data,
                             buf.ctypes.data, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data,
                             C.byref(est), None) == 1
    assert L.eifmm_ops_load(0, 1.0, 1, None, C.byref(h)) == 1
    assert L.eifmm_ops_build(0, 1.0, 3, -1.0, 100, None, C.byref(h)) == 1
    assert L.eifmm_evaluate(None, None, None, 0, 1, None, 0, 0, None) == 1
    assert L.eifmm_debug_export(None, 0, 2, None, 0) == 1
    # every other entry point rejects a null handle or output before any device work
    e, dk = C.c_double(), C.c_int()
    assert L.eifmm_ops_error_estimate(None, 2, C.byref(e), C.byref(dk)) == 1
    assert L.eifmm_ops_plan(None, 0, None) == 1
    assert L.eifmm_ops_calibrate(None, 1e-4, None, None) == 1
    assert L.eifmm_ops_calibration(None, None, None) == 1
    assert L.eifmm_tree_export(None, 0, None, None, None) == 1
    assert L.eifmm_evaluate_host(None, None, None, 0, 1, None, 0, 0, None) == 1
    assert L.eifmm_evaluate_batched(None, None, None, 0, None, 0, None) == 1
    assert L.eifmm_autotune(None, None, 1, 1, None, None) == 1
    assert L.eifmm_last_step_times(None, None) == 1
    assert L.eifmm_measure_rates(None, None) == 1
    assert L.eifmm_direct_sum(0, None, 0, None, 0, None, 0, 1, 0, None, 0, None, None) == 1
    L.eifmm_ops_destroy(None)
    L.eifmm_tree_destroy(None)


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    import importlib
    from paper_1408_0210_gb300 import eifmm as E
    monkeypatch.setattr(E, "_lib", None)
    monkeypatch.setattr(E, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        E.lib()
    importlib.reload(E)


def test_binding_rejects_bad_tensors_before_any_launch(E):
    """The binding checks dtype, shape, contiguity, device and output sizes of
    the static sort and the tree build before it calls the library: a float32
    or wrongly shaped array would make the kernels read past the buffer."""
    torch = pytest.importorskip("torch")
    n0 = E.eifmm_kernel_launches()
    bad = [
        (torch.zeros((10, 3), dtype=torch.float32), "float64"),
        (torch.zeros((10, 4), dtype=torch.float64), "shape"),
        (torch.zeros((3, 10), dtype=torch.float64).T, "contiguous"),
        (torch.zeros((10, 6), dtype=torch.float64)[:, :3], "contiguous"),
        (torch.zeros((10, 3), dtype=torch.float64), "CUDA"),
        (np.zeros((10, 3)), "torch tensor"),
    ]
    for x, msg in bad:
        with pytest.raises(ValueError, match=msg):
            E.eifmm_tree_sort_static(x, (0, 0, 0), 1.0, 3)
        with pytest.raises(ValueError, match=msg):
            E.eifmm_tree_build(x, None, (0, 0, 0), 1.0, 3, True)
    # output arrays: dtype, length and device, checked on their own
    dev = torch.device("cpu")
    with pytest.raises(ValueError, match="int32"):
        E.check_int32_out(torch.zeros(10, dtype=torch.int64), 10, dev, "keys")
    with pytest.raises(ValueError, match="at least 513"):
        E.check_int32_out(torch.zeros(512, dtype=torch.int32), 513, dev, "leaf_off")
    with pytest.raises(ValueError, match="contiguous"):
        E.check_int32_out(torch.zeros(40, dtype=torch.int32)[::2], 10, dev, "perm")
    with pytest.raises(ValueError, match="CUDA"):
        E.check_int32_out(torch.zeros(10, dtype=torch.int32), 10, dev, "perm")
    assert E.eifmm_kernel_launches() == n0


def test_tree_options_match_the_header(E):
    """The binding's option names and numbers are the header's
    EIFMM_OPT_* enumerators, and the entry point rejects a null tree, an
    unknown option and a value other than 0 or 1 before any device work."""
    txt = open(os.path.join(ROOT, "include", "eifmm.h")).read()
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"EIFMM_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    assert enum == E.OPTIONS
    L = E.lib()
    for opt in range(len(enum) + 2):
        assert L.eifmm_tree_set_option(None, opt, 1) == 1
    assert "unknown option" in L.eifmm_last_error().decode()


def test_binding_constants_match_the_header(E):
    """The binding's kernel, precision and status numbers and the static
    sort's point limit are the header's enumerators and define."""
    txt = open(os.path.join(ROOT, "include", "eifmm.h")).read()
    kern = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"EIFMM_KERNEL_([A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    assert kern == E.KERNELS
    prec = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"EIFMM_PREC_([A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    assert prec == E.PREC
    status = {int(m.group(2)): m.group(1) for m in re.finditer(r"EIFMM_(OK|E[A-Z]+)\s*=\s*(\d+)", txt)}
    assert status == E.STATUS
    lim = re.search(r"#define EIFMM_STATIC_SORT_MAX_POINTS (\d+)", txt)
    assert int(lim.group(1)) == E.STATIC_SORT_MAX_POINTS
