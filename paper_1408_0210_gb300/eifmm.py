"""Thin Python binding of the EIFMM C ABI (``include/eifmm.h``).

Every function here has the name of the C entry point it calls and only
marshals arguments (torch CUDA tensors or numpy arrays to pointers, status
codes to exceptions).  All arithmetic runs in ``libeifmm.so``; there is no
fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeifmm.so")

KERNELS = {"inv_r": 0, "config3": 1, "quad": 2, "one": 3, "exp_r2": 4,
           "cos20r_r": 5, "sqrt_r2p1": 6}
PREC = {"fp64": 0, "mixed": 1}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}
EXPORTS = [
    "eifmm_last_error", "eifmm_version", "eifmm_training_sets", "eifmm_eim_build",
    "eifmm_ops_load", "eifmm_ops_build", "eifmm_ops_error_estimate", "eifmm_ops_plan",
    "eifmm_ops_destroy", "eifmm_tree_build", "eifmm_tree_export", "eifmm_tree_destroy",
    "eifmm_evaluate", "eifmm_evaluate_host", "eifmm_evaluate_batched", "eifmm_debug_export",
    "eifmm_set_timing", "eifmm_last_step_times", "eifmm_direct_sum", "eifmm_kernel_launches",
    "eifmm_tree_sort_static", "eifmm_ops_calibrate", "eifmm_autotune", "eifmm_measure_rates",
    "eifmm_ops_calibration", "eifmm_tree_set_option", "eifmm_ops_compress", "eifmm_ops_basis",
    "eifmm_wait_selftest",
]
OPTIONS = {"m2l_128row": 0, "p2p_pair_symmetric": 1, "single_stream": 2, "m2l_fp64": 3,
           "m2l_stream_k": 4, "near_field_late": 5}


class EifmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LevelData(C.Structure):
    _fields_ = [("d", C.c_int), ("X", C.c_void_p), ("Y", C.c_void_p),
                ("Gamma", C.c_void_p), ("B", C.c_void_p), ("eps_est", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libeifmm.so (built in place by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "eifmm_last_error": (C.c_char_p, []),
        "eifmm_version": (C.c_char_p, []),
        "eifmm_training_sets": (i32, [i32, dbl, i32, vp, vp, vp, vp]),
        "eifmm_eim_build": (i32, [i32, vp, i64, vp, i64, dbl, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "eifmm_ops_load": (i32, [i32, dbl, i32, vp, vp]),
        "eifmm_ops_build": (i32, [i32, dbl, i32, dbl, i32, vp, vp]),
        "eifmm_ops_error_estimate": (i32, [vp, i32, vp, vp]),
        "eifmm_ops_plan": (i32, [vp, i32, vp]),
        "eifmm_ops_destroy": (None, [vp]),
        "eifmm_tree_build": (i32, [vp, i64, vp, i64, vp, dbl, i32, i32, vp, vp]),
        "eifmm_tree_export": (i32, [vp, i32, vp, vp, vp]),
        "eifmm_tree_destroy": (None, [vp]),
        "eifmm_evaluate": (i32, [vp, vp, vp, i64, i32, vp, i64, i32, vp]),
        "eifmm_evaluate_host": (i32, [vp, vp, vp, i64, i32, vp, i64, i32, vp]),
        "eifmm_autotune": (i32, [vp, vp, i32, i32, vp, vp]),
        "eifmm_measure_rates": (i32, [vp, vp]),
        "eifmm_evaluate_batched": (i32, [vp, vp, vp, i32, vp, i32, vp]),
        "eifmm_debug_export": (i32, [vp, i32, i32, vp, i64]),
        "eifmm_set_timing": (None, [i32]),
        "eifmm_last_step_times": (i32, [vp, vp]),
        "eifmm_direct_sum": (i32, [i32, vp, i64, vp, i64, vp, i64, i32, i32, vp, i64, vp, vp]),
        "eifmm_kernel_launches": (C.c_uint64, []),
        "eifmm_tree_sort_static": (i32, [vp, i64, vp, dbl, i32, vp, vp, vp, vp]),
        "eifmm_ops_calibrate": (i32, [vp, dbl, vp, vp]),
        "eifmm_ops_calibration": (i32, [vp, vp, vp]),
        "eifmm_tree_set_option": (i32, [vp, i32, i32]),
        "eifmm_ops_compress": (i32, [vp, dbl, vp, vp]),
        "eifmm_wait_selftest": (i32, [i64, vp]),
        "eifmm_ops_basis": (i32, [vp, i32, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise EifmmError(status, lib().eifmm_last_error().decode())


def _p(a) -> int | None:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _kid(kern) -> int:
    return KERNELS[kern] if isinstance(kern, str) else int(kern)


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def eifmm_version() -> str:
    return lib().eifmm_version().decode()


def eifmm_training_sets(level: int, L: float = 1.0, nJ: int = 9):
    nx, ny = C.c_int64(), C.c_int64()
    _check(lib().eifmm_training_sets(level, L, nJ, None, C.byref(nx), None, C.byref(ny)))
    X = np.zeros((nx.value, 3))
    Y = np.zeros((ny.value, 3))
    _check(lib().eifmm_training_sets(level, L, nJ, _p(X), C.byref(nx), _p(Y), C.byref(ny)))
    return X, Y


def eifmm_eim_build(kern, X, Y, eps: float, d_max: int = 512, stream=None) -> dict:
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    d = C.c_int()
    est = C.c_double()
    ia = np.zeros(d_max, dtype=np.int64)
    ib = np.zeros(d_max, dtype=np.int64)
    G = np.zeros((d_max, d_max))
    B = np.zeros((d_max, d_max))
    piv = np.zeros(d_max + 1)
    _check(lib().eifmm_eim_build(_kid(kern), _p(X), len(X), _p(Y), len(Y), float(eps), d_max,
                                 C.byref(d), _p(ia), _p(ib), _p(G), _p(B), _p(piv),
                                 C.byref(est), _stream(stream)))
    n = d.value
    return dict(d=n, ia=ia[:n].copy(), ib=ib[:n].copy(), Gamma=np.ascontiguousarray(G[:n, :n]),
                B=np.ascontiguousarray(B[:n, :n]), piv=piv[:n + 1].copy(), eps_est=est.value,
                X=X[ia[:n]].copy(), Y=Y[ib[:n]].copy())


class Ops:
    """Owner of an ``eifmm_ops`` handle."""

    def __init__(self, handle: int, depth: int, L: float):
        self.handle = handle
        self.depth = depth
        self.L = L

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.eifmm_ops_destroy(self.handle)
            self.handle = None

    def error_estimate(self, level: int):
        e, d = C.c_double(), C.c_int()
        _check(lib().eifmm_ops_error_estimate(self.handle, level, C.byref(e), C.byref(d)))
        return e.value, d.value

    def calibrate(self, eps: float, stream=None) -> int:
        t = C.c_int()
        _check(lib().eifmm_ops_calibrate(self.handle, float(eps), _stream(stream), C.byref(t)))
        return t.value

    def calibration(self) -> dict:
        """The last calibration: tier kept and the error of each tier
        evaluated (None where it was not)."""
        e, t = (C.c_double * 4)(), C.c_int()
        _check(lib().eifmm_ops_calibration(self.handle, e, C.byref(t)))
        return {"tier": t.value, "err": [v if v >= 0 else None for v in e]}

    def compress(self, eps: float, stream=None) -> dict:
        """eifmm_ops_compress: the M2L compression of Section 4.2 for the FP64
        far field (eps = 0 removes it); returns {level: rank}."""
        rk = (C.c_int * 11)()
        _check(lib().eifmm_ops_compress(self.handle, float(eps), _stream(stream), C.cast(rk, C.c_void_p)))
        return {k: rk[k] for k in range(2, self.depth + 1)}

    def basis(self, level: int) -> dict:
        """eifmm_ops_basis: U (d x r), the two filter counts and the singular
        values around the cut (relative to s_0)."""
        d, r = C.c_int(), C.c_int()
        info = (C.c_double * 4)()
        _check(lib().eifmm_ops_basis(self.handle, level, None, C.byref(d), C.byref(r), C.cast(info, C.c_void_p)))
        U = np.zeros((d.value, r.value))
        if r.value > 0:
            _check(lib().eifmm_ops_basis(self.handle, level, _p(U), None, None, None))
        return {"U": U, "d": d.value, "r": r.value, "r_i": int(info[0]), "r_ii": int(info[1]),
                "s_kept": info[2], "s_next": info[3]}

    def plan(self, tier_override: int = -1) -> int:
        t = C.c_int()
        _check(lib().eifmm_ops_plan(self.handle, tier_override, C.byref(t)))
        return t.value


def eifmm_ops_load(kern, L: float, depth: int, levels: dict) -> Ops:
    arr = (LevelData * (depth + 1))()
    keep = []
    for k in range(2, depth + 1):
        e = levels[k]
        parts = [np.ascontiguousarray(e[n], dtype=np.float64) for n in ("X", "Y", "Gamma", "B")]
        keep += parts
        arr[k] = LevelData(e["d"], *[p.ctypes.data for p in parts], float(e.get("eps_est", 0.0)))
    h = C.c_void_p()
    _check(lib().eifmm_ops_load(_kid(kern), float(L), depth, C.cast(arr, C.c_void_p), C.byref(h)))
    return Ops(h.value, depth, L)


def eifmm_ops_build(kern, L: float, depth: int, eps: float, d_max: int = 512, stream=None) -> Ops:
    h = C.c_void_p()
    _check(lib().eifmm_ops_build(_kid(kern), float(L), depth, float(eps), d_max, _stream(stream),
                                 C.byref(h)))
    return Ops(h.value, depth, L)


class Tree:
    """Owner of an ``eifmm_tree`` handle."""

    def __init__(self, handle: int, n_src: int, n_tgt: int, depth: int):
        self.handle = handle
        self.n_src = n_src
        self.n_tgt = n_tgt
        self.depth = depth
        self.p2p_pair_symmetric = None  # set by eifmm_autotune

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.eifmm_tree_destroy(self.handle)
            self.handle = None

    def set_option(self, name: str, value: bool) -> None:
        """eifmm_tree_set_option: one of OPTIONS, on (1) or off (0)."""
        _check(lib().eifmm_tree_set_option(self.handle, OPTIONS[name], int(bool(value))))

    def export(self, which: int = 0):
        n = self.n_src if which == 0 else self.n_tgt
        keys = np.zeros(n, dtype=np.uint32)
        perm = np.zeros(n, dtype=np.int32)
        off = np.zeros((1 << (3 * self.depth)) + 1, dtype=np.int64)
        _check(lib().eifmm_tree_export(self.handle, which, _p(keys), _p(perm), _p(off)))
        return keys, perm, off


def check_points(xyz, name: str = "xyz") -> None:
    """Raise ValueError unless xyz is a contiguous float64 (n, 3) CUDA tensor
    on the current device: the library reads 24 bytes per point from the
    current device's memory."""
    import torch
    if not isinstance(xyz, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if xyz.dtype != torch.float64:
        raise ValueError(f"{name}: dtype must be float64, not {xyz.dtype}")
    if xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError(f"{name}: shape must be (n, 3), not {tuple(xyz.shape)}")
    if not xyz.is_contiguous():
        raise ValueError(f"{name}: must be contiguous (row-major n x 3)")
    if not xyz.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if xyz.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {xyz.device}, but the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def check_int32_out(t, min_len: int, device, name: str) -> None:
    """Raise ValueError unless t is a contiguous int32 CUDA tensor on `device`
    with at least min_len elements (the library writes that many)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if t.dtype != torch.int32:
        raise ValueError(f"{name}: dtype must be int32, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() < min_len:
        raise ValueError(f"{name}: needs at least {min_len} elements, has {t.numel()}")
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name}: must be a CUDA tensor on {device}, not {t.device}")


def eifmm_tree_build(src_xyz, tgt_xyz=None, lo=(0.0, 0.0, 0.0), L: float = 1.0, depth: int = 3,
                     exclude_self: bool = True, stream=None) -> Tree:
    """src_xyz / tgt_xyz: CUDA float64 tensors of shape (n, 3), contiguous,
    on the current device."""
    tgt = src_xyz if tgt_xyz is None else tgt_xyz
    check_points(src_xyz, "src_xyz")
    check_points(tgt, "tgt_xyz")
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    h = C.c_void_p()
    _check(lib().eifmm_tree_build(_p(src_xyz), src_xyz.shape[0], _p(tgt), tgt.shape[0], _p(lo),
                                  float(L), depth, int(bool(exclude_self)), _stream(stream),
                                  C.byref(h)))
    return Tree(h.value, src_xyz.shape[0], tgt.shape[0], depth)


def eifmm_evaluate(tree: Tree, ops: Ops, sigma, f, prec="fp64", stream=None) -> None:
    """sigma (n_src, R) and f (n_tgt, R): CUDA float64 tensors, column-major
    (use ``t.T.contiguous().T`` or allocate as ``torch.empty(R, n).T``).
    sigma must be finite: the mixed path's M2M/L2L library GEMMs do not carry
    infinities or NaNs through."""
    import torch
    for name, t, n in (("sigma", sigma, tree.n_src), ("f", f, tree.n_tgt)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError(f"{name}: a float64 CUDA tensor is required")
        if t.dim() not in (1, 2) or t.shape[0] != n:
            raise ValueError(f"{name}: needs {n} rows, has shape {tuple(t.shape)}")
    R = 1 if sigma.dim() == 1 else sigma.shape[1]
    if (1 if f.dim() == 1 else f.shape[1]) != R:
        raise ValueError("sigma and f need the same number of columns")
    ld_s = sigma.shape[0] if sigma.dim() == 1 or R == 1 else sigma.stride(1)
    ld_f = f.shape[0] if f.dim() == 1 or R == 1 else f.stride(1)
    if (sigma.dim() == 1 or R == 1) and not (sigma.is_contiguous() and f.is_contiguous()):
        raise ValueError("sigma and f must be contiguous")
    if R > 1 and not (sigma.stride(0) == 1 and f.stride(0) == 1):
        raise ValueError("sigma and f must be column-major")
    _check(lib().eifmm_evaluate(tree.handle, ops.handle, _p(sigma), ld_s, R, _p(f), ld_f,
                                _prec(prec), _stream(stream)))


def eifmm_evaluate_host(tree: Tree, ops: Ops, sigma, f=None, prec="fp64", stream=None):
    """HOST float64 arrays (n, R), column-major; returns f."""
    sigma = np.asfortranarray(sigma if np.ndim(sigma) == 2 else np.asarray(sigma)[:, None],
                              dtype=np.float64)
    R = sigma.shape[1]
    if f is None:
        f = np.zeros((tree.n_tgt, R), order="F")
    _check(lib().eifmm_evaluate_host(tree.handle, ops.handle, _p(sigma), sigma.shape[0], R, _p(f),
                                     f.shape[0], _prec(prec), _stream(stream)))
    return f


def eifmm_evaluate_batched(trees, sigmas, fs, ops: Ops, prec="fp64", stream=None) -> None:
    n = len(trees)
    th = (C.c_void_p * n)(*[t.handle for t in trees])
    sp = (C.c_void_p * n)(*[_p(s) for s in sigmas])
    fp = (C.c_void_p * n)(*[_p(x) for x in fs])
    _check(lib().eifmm_evaluate_batched(C.cast(th, C.c_void_p), C.cast(sp, C.c_void_p),
                                        C.cast(fp, C.c_void_p), n, ops.handle, _prec(prec),
                                        _stream(stream)))


def eifmm_measure_rates(stream=None) -> dict:
    """Measured FP32 FMA/s, approximate rsqrt/s and FP64 FMA/s of this GPU."""
    r = (C.c_double * 3)()
    _check(lib().eifmm_measure_rates(_stream(stream), C.cast(r, C.c_void_p)))
    return {"ffma_per_s": r[0], "rsqrt_per_s": r[1], "dfma_per_s": r[2]}


M2L_VARIANTS = {0: "rule", 1: "transposed", 2: "128-row", 3: "transposed stream-K"}


def eifmm_autotune(tree: Tree, ops: Ops, n_rhs: int = 1, prec="mixed", stream=None) -> dict:
    """Time the M2L variants per level on this tree and keep the fastest;
    returns {level: (variant, group shift)}.  The near-field kernel chosen by
    the same timing is left in tree.p2p_pair_symmetric (True when the
    pair-symmetric near field was kept)."""
    ch = (C.c_int * 22)()
    _check(lib().eifmm_autotune(tree.handle, ops.handle, int(n_rhs), _prec(prec), _stream(stream),
                                C.cast(ch, C.c_void_p)))
    tree.p2p_pair_symmetric = bool(ch[0])
    return {k: (ch[2 * k], ch[2 * k + 1]) for k in range(2, tree.depth + 1)}


def eifmm_debug_export(tree: Tree, what: int, level: int, d: int, R: int = 1):
    if what in (5, 6):
        out = np.zeros(tree.n_tgt * R)
        _check(lib().eifmm_debug_export(tree.handle, what, level, _p(out), out.size))
        return out.reshape(R, tree.n_tgt).T.copy()
    out = np.zeros((8 ** level, R, d))
    _check(lib().eifmm_debug_export(tree.handle, what, level, _p(out), out.size))
    return out


def eifmm_set_timing(on: bool) -> None:
    lib().eifmm_set_timing(int(bool(on)))


def eifmm_last_step_times(tree: Tree) -> list[float]:
    ms = (C.c_float * 20)()
    _check(lib().eifmm_last_step_times(tree.handle, C.cast(ms, C.c_void_p)))
    return list(ms)


def eifmm_direct_sum(kern, tgt_xyz, src_xyz, sigma, exclude_self=True, tgt_idx=None, stream=None):
    """Exact FP64 sum on the GPU at the targets tgt_idx (CUDA int64) or all
    targets; sigma (n_src,) or column-major (n_src, R).  Returns f (n_eval, R)."""
    import torch
    R = 1 if sigma.dim() == 1 else sigma.shape[1]
    ld = sigma.shape[0] if (sigma.dim() == 1 or R == 1) else sigma.stride(1)
    n_eval = tgt_xyz.shape[0] if tgt_idx is None else tgt_idx.shape[0]
    f = torch.zeros(R, n_eval, dtype=torch.float64, device=sigma.device).T
    _check(lib().eifmm_direct_sum(_kid(kern), _p(tgt_xyz), tgt_xyz.shape[0], _p(src_xyz),
                                  src_xyz.shape[0], _p(sigma), ld, R, int(bool(exclude_self)),
                                  _p(tgt_idx), n_eval, _p(f), _stream(stream)))
    return f


def eifmm_wait_selftest(limit_cycles: int) -> tuple[int, int]:
    """Runs the library's bounded device wait on a barrier nothing completes;
    returns (status, code): (4 = ETIMEOUT, 7) when the wait gave up."""
    code = C.c_int(-1)
    st = lib().eifmm_wait_selftest(int(limit_cycles), C.byref(code))
    return st, code.value


def eifmm_kernel_launches() -> int:
    return int(lib().eifmm_kernel_launches())


STATIC_SORT_MAX_POINTS = 1048576


def eifmm_tree_sort_static(xyz, lo=(0.0, 0.0, 0.0), L: float = 1.0, depth: int = 3,
                           keys=None, perm=None, leaf_off=None, stream=None):
    """Allocation-free bin/sort into caller-owned CUDA tensors (created here
    when not given): returns (keys uint32 as int32 bits, perm int32,
    leaf_off int32).  xyz: contiguous float64 (n, 3) CUDA tensor on the
    current device; keys and perm: int32, at least n entries; leaf_off:
    int32, at least 8^depth + 1 entries; all on xyz's device.  Invalid
    arguments raise ValueError before anything runs on the GPU."""
    import torch
    check_points(xyz, "xyz")
    if not (2 <= int(depth) <= 10):
        raise ValueError(f"depth must lie in [2, 10], not {depth}")
    n = xyz.shape[0]
    dev = xyz.device
    for name, t, need in (("keys", keys, n), ("perm", perm, n), ("leaf_off", leaf_off, (1 << (3 * depth)) + 1)):
        if t is not None:
            check_int32_out(t, need, dev, name)
    if keys is None:
        keys = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if perm is None:
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if leaf_off is None:
        leaf_off = torch.empty((1 << (3 * depth)) + 1, dtype=torch.int32, device=dev)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    _check(lib().eifmm_tree_sort_static(_p(xyz), n, _p(lo), float(L), depth, _p(keys), _p(perm),
                                        _p(leaf_off), _stream(stream)))
    return keys[:n], perm[:n], leaf_off
