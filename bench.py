#!/usr/bin/env python3
"""Throughput of the EIFMM evaluation (Algorithm 3 steps 1-7 + near field +
un-permute) on one GB300, in targets x RHS per second.

Workload: 1,048,576 points iid uniform in [0,1)^3 (targets = sources, self pair
excluded), K(r) = 1/|r|, octree depth 5 (32,768 leaves, 32 points per leaf),
one sigma vector iid U[-1,1]; operators from the GPU EIM at eps = 1e-4 and
eps = 1e-7.  One step = one eifmm_evaluate call with sigma and f resident in
HBM; the tree is built and the operators loaded beforehand.  Between timed
steps a 512 MB buffer is written to flush the 129 MB L2.

Every variant's accuracy is checked against the exact FP64 sum (the library's
GPU direct sum) on 2048 sampled targets; `value` is the mixed-precision path at
eps = 1e-4 when it meets rel-L2 <= eps, else the FP64 path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the CPU checker of the repository (plain FP64 C, OpenMP)
runs the same metric on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "targets*RHS/s (EIFMM evaluate, rel-L2 <= eps)"
UNIT = "targets*RHS/s"
N_POINTS = 1 << 20
DEPTH = 5
NRHS = 1
EPS_LIST = (1e-4, 1e-7)
SAMPLE_TARGETS = 2048
WORKLOAD = "uniform cube N=1048576, K=1/r, depth 5, 1 RHS"


def m2l_pairs(k: int) -> int:
    """Exact number of (I, J) interaction-list pairs at level k (separable)."""
    n = 1 << k
    sa = sum(min(n - 1, 2 * (i >> 1) + 3) - max(0, 2 * (i >> 1) - 2) + 1 for i in range(n))
    sb = sum(min(n - 1, i + 1) - max(0, i - 1) + 1 for i in range(n))
    return sa ** 3 - sb ** 3


def near_field_pairs(off: np.ndarray, depth: int) -> int:
    """Exact source-target pairs of the near field: every target against the
    points of the 27 leaves around its own, minus the self pairs."""
    n = 1 << depth
    cnt = np.diff(off).astype(np.int64)
    key = np.arange(cnt.size, dtype=np.int64)
    c = np.zeros((3, cnt.size), dtype=np.int64)
    for b in range(depth):
        for a in range(3):
            c[a] |= ((key >> (3 * b + a)) & 1) << b
    grid = np.zeros((n + 2, n + 2, n + 2), dtype=np.int64)
    grid[c[2] + 1, c[1] + 1, c[0] + 1] = cnt
    nb = sum(grid[1 + dz:n + 1 + dz, 1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx]
             for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    own = grid[1:n + 1, 1:n + 1, 1:n + 1]
    return int((own * nb).sum() - cnt.sum())


# one ncu capture of the level-5 k_m2l_t256 launch (dram read + write bytes)
M2L_T256_TRAFFIC = 37.545728e6 + 0.145408e6
# nominal special-function rate: 16 results per clock per SM, 152 SMs, 2070 MHz
SFU_PEAK = 16 * 152 * 2.07e9


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group("nccl")
    return rank, ws, dist


def max_over_ranks(ms: float, dist, device="cuda") -> float:
    """The job's step time: the slowest rank's (each rank runs its own
    replica of the workload, no data-path collective)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world_size: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's
    step time."""
    return units_per_rank * world_size / (ms * 1e-3)


def cpu_oracle_run(n: int, depth: int, eps: float, steps: int, warmup: int = 0):
    """Time the CPU checker's EIFMM (O2) on n points after `warmup` untimed
    evaluations; returns (seconds per evaluation, threads, d per level)."""
    import oracle
    from paper_1408_0210_gb300 import workloads as wl
    x = wl.uniform_cube(n, 2)
    s = wl.sigma_uniform(n, NRHS, 102)
    lv = oracle.build_levels("inv_r", 1.0, depth, eps)
    for _ in range(warmup):
        oracle.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv, x, x, s)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.eifmm("inv_r", 1.0, [0, 0, 0], depth, lv, x, x, s)
        times.append(time.perf_counter() - t0)
    return statistics.median(times), oracle.num_threads(), [lv[k]["d"] for k in sorted(lv)]


# the bounded CPU sample: 131,072 points at depth 4 keeps 32 points per leaf
CPU_SAMPLE_N, CPU_SAMPLE_DEPTH = 1 << 17, 4
CPU_SAMPLE_WORKLOAD = (f"uniform cube N={CPU_SAMPLE_N} (bounded sample of the N={N_POINTS} workload), "
                       f"K=1/r, depth {CPU_SAMPLE_DEPTH} (32 points/leaf as in the workload), {NRHS} RHS")


def reference_arm(args):
    rank, ws, dist = (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), None)
    if rank != 0:
        return
    eps = EPS_LIST[0]
    sec, threads, ds = cpu_oracle_run(CPU_SAMPLE_N, CPU_SAMPLE_DEPTH, eps, max(1, args.steps),
                                      max(args.warmup, 0))
    value = CPU_SAMPLE_N * NRHS / sec
    sample = (f"CPU EIFMM (plain FP64 C + OpenMP) on {CPU_SAMPLE_N} uniform points at depth "
              f"{CPU_SAMPLE_DEPTH} (32 points/leaf as in the workload), eps={eps:g}, d={ds}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": CPU_SAMPLE_WORKLOAD, "eps": eps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# The other workloads: timed the same way (CUDA events on the launching
# stream, a 512 MB write between steps), each with its accuracy against the
# exact FP64 sum on sampled targets (the worst right-hand side).
# --------------------------------------------------------------------------
WORKLOADS = {
    "c1": "uniform cube N=4096, K=1/r, depth 3, eps 1e-6, 1 RHS, FP64 path",
    "c3": ("8-Gaussian mixture N=1048576 (std 0.05, centres U[0.2,0.8]^3, clipped), "
           "K=exp(-r)/r + 1/sqrt(r1^2+0.01 r2^2+r3^2+1e-3), depth 5, eps 1e-6, 1 RHS, mixed"),
    "c4a": "uniform cube N=262144, K=1/r, depth 5, eps 1e-6, 64 RHS, mixed",
    "c4a+c": ("uniform cube N=262144, K=1/r, depth 5, eps 1e-6, 64 RHS, mixed, M2L compressed "
              "(Section 4.2 first stage)"),
    "c4b": ("32 problems, N log-uniform in [16384, 262144], own uniform points and trees "
            "(depth clamp(ceil(log8(N/32)), 3, 5)), one operator set, K=1/r, eps 1e-6, "
            "one graph launch, mixed"),
    "c5": "uniform cube N=16777216, K=1/r, depth 7, eps 1e-5, 8 RHS N(0,1), mixed",
    "sphere": "sphere surface r=0.5, N=992046, K=1/r, depth 7, eps 1e-4, 1 RHS, mixed",
}


def run_workloads(names, stream, flush, dist, profile_steps=0):
    import math

    import torch

    from paper_1408_0210_gb300 import eifmm as E
    from paper_1408_0210_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())

    def cols(s):
        return torch.from_numpy(np.asfortranarray(s)).to(dev).T.contiguous().T

    def timed(fn, steps, warmup, st=stream):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if profile_steps > 0:  # for ncu --profile-from-start off: no timing
            torch.cuda.profiler.start()
            for _ in range(profile_steps):
                with torch.cuda.stream(st):
                    fn()
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            return float("nan"), 0
        launches0 = E.eifmm_kernel_launches()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        for i in range(steps):
            with torch.cuda.stream(st):
                flush.zero_()
                e0[i].record(st)
                fn()
                e1[i].record(st)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / steps
        return max_over_ranks(ms, dist, dev), (E.eifmm_kernel_launches() - launches0) // steps

    def err_vs_exact(kern, x, s, f, idx):
        xd = torch.from_numpy(x).to(dev)
        ref = E.eifmm_direct_sum(kern, xd, xd, cols(s), True, torch.from_numpy(idx).to(dev), stream)
        got = f[torch.from_numpy(idx).to(dev)]
        num = torch.linalg.norm(got - ref, dim=0) / torch.linalg.norm(ref, dim=0)
        return float(num.max())

    out = {}
    for name in names:
        r = {"workload": WORKLOADS[name]}
        try:
            if name in ("c1", "c3", "c4a", "c4a+c", "c5", "sphere"):
                kern, n, depth, eps, R, prec, steps, warmup = {
                    "c1": ("inv_r", 4096, 3, 1e-6, 1, "fp64", 10, 3),
                    "c3": ("config3", 1 << 20, 5, 1e-6, 1, "mixed", 3, 3),
                    "c4a": ("inv_r", 262144, 5, 1e-6, 64, "mixed", 1, 1),
                    "c4a+c": ("inv_r", 262144, 5, 1e-6, 64, "mixed", 1, 1),
                    "c5": ("inv_r", 1 << 24, 7, 1e-5, 8, "mixed", 2, 3),
                    "sphere": ("inv_r", 992046, 7, 1e-4, 1, "mixed", 5, 3),
                }[name]
                x = {"c1": lambda: wl.uniform_cube(n, 1), "c3": lambda: wl.gaussian_mixture(n, 3),
                     "c4a": lambda: wl.uniform_cube(n, 4), "c4a+c": lambda: wl.uniform_cube(n, 4),
                     "c5": lambda: wl.uniform_cube(n, 5),
                     "sphere": lambda: wl.sphere_surface(n, 6)}[name]()
                s = (wl.sigma_normal(n, R, 105) if name == "c5" else
                     wl.sigma_uniform(n, R, {"c1": 101, "c3": 103, "c4a": 104, "c4a+c": 104, "sphere": 106}[name]))
                ops = E.eifmm_ops_build(kern, 1.0, depth, eps, 512, stream)
                if name.endswith("+c"):
                    r["m2l_rank"] = ops.compress(eps, stream)
                tree = E.eifmm_tree_build(torch.from_numpy(x).to(dev), None, (0, 0, 0), 1.0, depth, True, stream)
                sd = cols(s) if R > 1 else torch.from_numpy(np.ascontiguousarray(s[:, 0])).to(dev)
                f = (torch.zeros(R, n, dtype=torch.float64, device=dev).T if R > 1
                     else torch.zeros(n, dtype=torch.float64, device=dev))
                if prec == "mixed" and ops.plan() <= 1:
                    E.eifmm_autotune(tree, ops, R, prec, stream)
                ms, launches = timed(lambda: E.eifmm_evaluate(tree, ops, sd, f, prec, stream), steps, warmup)
                # the 16M-point workload is checked on 4096 random targets
                idx = wl.sample_targets(n, 4096 if name == "c5" else (512 if R == 1 else 128), 55)
                ff = f if R > 1 else f[:, None]
                r.update({"n_targets": n, "n_rhs": R, "eps": eps, "path": prec,
                          "tier": ops.plan() if prec == "mixed" else None,
                          "d": [ops.error_estimate(k)[1] for k in range(2, depth + 1)],
                          "ms_per_step": ms, "steps": steps, "warmup": warmup, "gpu_launches": launches,
                          "value": n * R / (ms * 1e-3), "unit": UNIT,
                          "rel_l2_vs_exact": err_vs_exact(kern, x, s, ff, idx), "sampled_targets": len(idx)})
                if name == "c3":
                    r["note"] = ("the anisotropic kernel is not well separated across boxes split only "
                                 "along y, so the method stays near 1e-1 of the exact sum (FP64 path too)")
                del tree, ops, sd, f, ff
            elif name == "c4b":
                eps = 1e-6
                sizes = wl.batch_sizes(32, 16384, 262144, 40)
                depths = [min(5, max(3, math.ceil(math.log(nn / 32, 8)))) for nn in sizes]
                ops = E.eifmm_ops_build("inv_r", 1.0, max(depths), eps, 512, stream)
                xs = [wl.uniform_cube(nn, 40 + p) for p, nn in enumerate(sizes)]
                ss = [wl.sigma_uniform(nn, 1, 140 + p) for p, nn in enumerate(sizes)]
                trees = [E.eifmm_tree_build(torch.from_numpy(xx).to(dev), None, (0, 0, 0), 1.0, d, True, stream)
                         for xx, d in zip(xs, depths)]
                sd = [torch.from_numpy(np.ascontiguousarray(q[:, 0])).to(dev) for q in ss]
                fb = [torch.zeros(nn, dtype=torch.float64, device=dev) for nn in sizes]
                # a stream of its own: the batched call records its graph on the
                # first call and replays it with one launch afterwards (the
                # legacy default stream is never captured)
                s2 = torch.cuda.Stream()
                ms, launches = timed(lambda: E.eifmm_evaluate_batched(trees, sd, fb, ops, "mixed", s2), 3, 3, s2)
                errs = []
                for p in (0, 7, 19, 31):
                    idx = wl.sample_targets(sizes[p], 256, 200 + p)
                    errs.append(err_vs_exact("inv_r", xs[p], ss[p], fb[p][:, None], idx))
                r.update({"n_targets": int(sum(sizes)), "n_problems": 32, "n_rhs": 1, "eps": eps, "path": "mixed",
                          "tier": ops.plan(), "ms_per_step": ms, "steps": 3, "warmup": 3,
                          "gpu_launches_host_side": launches,
                          "note": "after the first call every step is one CUDA-graph launch of the 32 evaluations",
                          "value": sum(sizes) / (ms * 1e-3), "unit": UNIT,
                          "rel_l2_vs_exact": max(errs), "sampled_problems": [0, 7, 19, 31]})
                del trees, ops, sd, fb
        except Exception as e:  # report, keep the other workloads
            r["unavailable"] = f"{type(e).__name__}: {e}"
        out[name] = r
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="mixed:1e-4,fp64:1e-4,mixed:1e-5,mixed:1e-6,mixed+c:1e-6,fp64:1e-6,fp64+c:1e-6,mixed:1e-7,fp64:1e-7")
    ap.add_argument("--workloads", default="c1,c3,c4a,c4a+c,c4b,c5,sphere",
                    help="other benchmark workloads to time after the headline ('' for none)")
    ap.add_argument("--tree-option", action="append", default=[],
                    help="name=0|1: eifmm_tree_set_option on the workload's tree (for comparisons)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in M2L and near-field rules (with --tree-option, to compare kernels)")
    ap.add_argument("--profile-workload-steps", type=int, default=0,
                    help="run this many evaluations of each --workloads entry between "
                         "cudaProfilerStart/Stop instead of timing them")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run this many evaluations of the first variant between "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off) and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    args.warmup = max(args.warmup, 3)

    import torch

    from paper_1408_0210_gb300 import eifmm as E
    from paper_1408_0210_gb300 import workloads as wl

    rank, ws, dist = dist_setup()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    pk = peaks()
    rates = E.eifmm_measure_rates(stream)  # FP32 FMA, approximate rsqrt, FP64 FMA per second

    # ---- inputs (per rank: an independent replica of the workload) -------
    x = wl.uniform_cube(N_POINTS, 2 + 1000 * rank)
    s = wl.sigma_uniform(N_POINTS, NRHS, 102 + 1000 * rank)
    xd = torch.from_numpy(x).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(s[:, 0])).to(dev)
    f = torch.zeros(N_POINTS, dtype=torch.float64, device=dev)
    tree = E.eifmm_tree_build(xd, None, (0, 0, 0), 1.0, DEPTH, True, stream)
    for opt in args.tree_option:
        name, val = opt.split("=")
        tree.set_option(name, val not in ("0", "false", "False"))
    # the tree build (step a0, outside the timed evaluate as in the paper),
    # timed on its own: device events around a few rebuilds
    tb = []
    for i in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tt = E.eifmm_tree_build(xd, None, (0, 0, 0), 1.0, DEPTH, True, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            tb.append(e0.elapsed_time(e1))
        del tt
    tree_ms = statistics.median(tb)
    idx = torch.from_numpy(wl.sample_targets(N_POINTS, SAMPLE_TARGETS, 55)).to(dev)
    fref = E.eifmm_direct_sum("inv_r", xd, xd, sd, True, idx, stream)[:, 0]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    # a variant: path (fp64 / mixed), EIM tolerance, and "+c" for the M2L
    # compression of Section 4.2 (its own operator set: the FP64 far field
    # runs the compressed M2L)
    variants = []
    for v in args.variants.split(","):
        name, eps = v.split(":")
        variants.append((name, float(eps)))
    ops = {}
    ops_err = {}
    for name, eps in variants:
        key = (eps, name.endswith("+c"))
        if key not in ops and key not in ops_err:
            try:
                ops[key] = E.eifmm_ops_build("inv_r", 1.0, DEPTH, eps, 512, stream)
                if key[1]:
                    ops[key].compress(eps, stream)
            except E.EifmmError as e:
                ops_err[key] = str(e)

    if args.profile_steps > 0:
        name, eps = variants[0]
        prec, o = name.split("+")[0], ops[(eps, name.endswith("+c"))]
        if prec == "mixed" and not args.no_autotune:
            E.eifmm_autotune(tree, o, NRHS, prec, stream)
        for _ in range(max(args.warmup, 1)):
            E.eifmm_evaluate(tree, o, sd, f, prec, stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.profile_steps):
            E.eifmm_evaluate(tree, o, sd, f, prec, stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return

    def run_variant(name, eps, steps, warmup, timing=False):
        prec, o = name.split("+")[0], ops[(eps, name.endswith("+c"))]
        tuned = None
        if prec == "mixed" and not args.no_autotune:
            # the M2L autotuner (setup, like the tree build): per-level variant
            tuned = E.eifmm_autotune(tree, o, NRHS, prec, stream)
        for _ in range(warmup):
            E.eifmm_evaluate(tree, o, sd, f, prec, stream)
        torch.cuda.synchronize()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        E.eifmm_set_timing(timing)
        step_times = []
        launches0 = E.eifmm_kernel_launches()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            e0[i].record(stream)
            E.eifmm_evaluate(tree, o, sd, f, prec, stream)
            e1[i].record(stream)
            if timing:
                step_times.append(E.eifmm_last_step_times(tree))
        torch.cuda.synchronize()
        launches = E.eifmm_kernel_launches() - launches0
        E.eifmm_set_timing(False)
        ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / steps
        ms = max_over_ranks(ms, dist, dev)
        err = float(torch.linalg.norm(f[idx] - fref) / torch.linalg.norm(fref))
        return ms, err, launches, step_times, tuned

    results = {}
    headline = None
    with ClockSampler(torch.cuda.current_device()) as clk:
        for name, eps in variants:
            prec, key = name.split("+")[0], (eps, name.endswith("+c"))
            if key in ops_err:
                results[f"{name}@{eps:g}"] = {"unavailable": ops_err[key]}
                continue
            try:
                steps = args.steps if (prec == "mixed" or eps >= 1e-5) else max(3, args.steps // 3)
                ms, err, launches, st, tuned = run_variant(name, eps, steps, args.warmup, timing=True)
            except E.EifmmError as e:
                results[f"{name}@{eps:g}"] = {"unavailable": str(e)}
                continue
            o = ops[key]
            d = [o.error_estimate(k)[1] for k in range(2, DEPTH + 1)]
            m2l = [statistics.median([t[9 + k] for t in st]) for k in range(2, DEPTH + 1)]
            results[f"{name}@{eps:g}"] = {
                "value": job_throughput(N_POINTS * NRHS, ws, ms), "ms_per_step": ms,
                "tier": o.plan() if prec == "mixed" else None,
                "calibration": o.calibration() if prec == "mixed" else None,
                "m2l_rank": ({str(k): o.basis(k)["r"] for k in range(2, DEPTH + 1)} if key[1] else None),
                "rel_l2_vs_exact": err, "meets_eps": err <= eps, "d": d,
                "gpu_launches": launches, "steps": steps,
                "step_ms": [round(statistics.median([t[i] for t in st]), 4) for i in range(8)],
                "nf_ms": round(statistics.median([t[8] for t in st]), 4),
                "m2l_autotune": ({str(k): [E.M2L_VARIANTS[v], g] for k, (v, g) in tuned.items()}
                                 if tuned else None),
                "p2p_pair_symmetric": tree.p2p_pair_symmetric if tuned else None,
                "m2l_ms_per_level": [round(v, 4) for v in m2l]}
            if headline is None and err <= eps and (name, eps) in (("mixed", 1e-4), ("fp64", 1e-4)):
                headline = (name, eps)
        names = [w for w in args.workloads.split(",") if w]
        workloads = run_workloads(names, stream, flush, dist, args.profile_workload_steps) if names else {}
    clocks = clk.summary()

    if headline is None:  # no 1e-4 variant met its tolerance: the first one that ran
        headline = next(((p, e) for p, e in variants if "value" in results.get(f"{p}@{e:g}", {})),
                        variants[0])
    hp, he = headline
    hr = results[f"{hp}@{he:g}"]

    # ---- end to end through the host-buffer entry point -------------------
    sh = torch.from_numpy(np.ascontiguousarray(s[:, 0])).pin_memory()
    fh = torch.zeros(N_POINTS, dtype=torch.float64).pin_memory()
    for _ in range(2):
        E.lib().eifmm_evaluate_host(tree.handle, ops[(he, False)].handle, sh.data_ptr(), N_POINTS, 1,
                                    fh.data_ptr(), N_POINTS, E.PREC[hp], stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ke = max(3, args.steps // 2)
    for _ in range(ke):
        rc = E.lib().eifmm_evaluate_host(tree.handle, ops[(he, False)].handle, sh.data_ptr(), N_POINTS, 1,
                                         fh.data_ptr(), N_POINTS, E.PREC[hp], stream.cuda_stream)
        assert rc == 0, E.lib().eifmm_last_error()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / ke * 1e3, dist, dev)
    e2e_val = job_throughput(N_POINTS * NRHS, ws, e2e_ms)

    # ---- roofline of the dominant kernel: the M2L of the leaf level ------
    o = ops[(he, False)]
    dk = o.error_estimate(DEPTH)[1]
    flops = 2.0 * dk * dk * m2l_pairs(DEPTH) * NRHS
    m2l_ms = hr["m2l_ms_per_level"][-1]
    achieved = flops / (m2l_ms * 1e-3) / 1e12
    if hp == "mixed":
        # the tensor pipe does more than the algorithmic work: 3 split products
        # (hi*hi, hi*lo, lo*hi), the padding of d to dp, and the 189 candidate
        # offsets of a parity class against the pairs that exist
        dp = (dk + 63) // 64 * 64
        issued = 3.0 * (dp / dk) ** 2 * (189 * 8 ** DEPTH) / m2l_pairs(DEPTH)
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"],
                "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
                "traffic": M2L_T256_TRAFFIC if dk <= 128 else None,
                "kernel": "M2L level 5 (k_m2l_t256: tcgen05 M=128 x N=256, BF16 split operands, FP32 accumulate)",
                "peak_source": pk["source"] + " bf16 burst",
                "issued_over_algorithmic": issued,
                "issued_frac": achieved * issued / pk["bf16_tflops"],
                "issued_note": "derived: tensor work issued = algorithmic x issued_over_algorithmic"}
    else:
        peak64 = 2.0 * rates["dfma_per_s"] / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                "frac": achieved / peak64, "traffic": None,
                "kernel": "M2L level 5 (FP64 FMA)", "peak_source": "measured FP64 FMA register loop"}

    # ---- second bound: the near field, one approximate 1/r per pair ----------
    _, _, off = tree.export(1)
    pairs = near_field_pairs(off, DEPTH)
    nf_ms = hr["nf_ms"]
    roof_nf = None
    if nf_ms > 0:
        rs = rates["rsqrt_per_s"]
        # tier 0 with one right-hand side visits each unordered leaf pair once:
        # one 1/r per unordered point pair, the own leaf in full
        sym = False  # the per-target near field (the pair-symmetric one is an option of the tree)
        cnt = np.diff(off).astype(np.int64)
        own = int((cnt * (cnt - 1)).sum())
        evals = (pairs - own) // 2 + own if sym else pairs
        name = ("k_p2p32_sym, FP32, each leaf pair once" if sym else
                "k_p2p32x, FP32, packed distances" if hp == "mixed" else "k_p2p64, FP64")
        roof_nf = {"bound": "alu", "achieved": evals / (nf_ms * 1e-3), "peak": rs,
                   "unit": "rsqrt/s", "frac": evals / (nf_ms * 1e-3) / rs, "traffic": None,
                   "kernel": f"near field ({name}), {pairs} directed pairs, {evals} 1/r evaluations",
                   "pairs_per_s": pairs / (nf_ms * 1e-3), "launch_ms": nf_ms,
                   "note": ("the near field runs at the lowest stream priority beside the far field, "
                            "so launch_ms is its wall span inside the step, not its cost alone"),
                   "peak_source": "measured rsqrt.approx register loop",
                   "nominal_peak": SFU_PEAK}

    acc_ref = {"kind": "exact FP64 sum of Eq. (1) on the GPU (eifmm_direct_sum), self pair excluded",
               "targets": SAMPLE_TARGETS}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sec, threads, ds = cpu_oracle_run(CPU_SAMPLE_N, CPU_SAMPLE_DEPTH, he, 1)
        cpu = {"value": CPU_SAMPLE_N * NRHS / sec, "unit": UNIT, "cores": threads,
               "kind": "oracle",
               "sample": f"CPU EIFMM (plain FP64 C + OpenMP) on {CPU_SAMPLE_N} uniform points, "
                         f"depth {CPU_SAMPLE_DEPTH} (32 points/leaf), eps={he:g}, d={ds}"}
        # the accuracy reference itself (the GPU exact sum) against the CPU
        # oracle's exact sum O1 on the first 256 sampled targets
        import oracle
        i256 = idx[:256].cpu().numpy()
        o1 = oracle.direct_sum("inv_r", x, x, s, exclude_self=True, tgt_idx=i256)[:, 0]
        g1 = fref[:256].cpu().numpy()
        acc_ref["max_rel_diff_vs_cpu_oracle_exact_sum"] = float(np.max(np.abs(g1 - o1)) / np.max(np.abs(o1)))
        acc_ref["oracle_targets"] = 256

    line = {
        "metric": METRIC, "value": hr["value"], "unit": UNIT, "n_gpus": ws,
        "steps": hr["steps"], "warmup": args.warmup, "ms_per_step": hr["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+bf16x3" if hp == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "eps": he, "path": hp, "l2": "flushed (512 MB write) between steps",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": N_POINTS * NRHS * 8,
                "d2h_bytes_per_step": N_POINTS * NRHS * 8},
        "gpu_launches": hr["gpu_launches"],
        "accuracy_reference": acc_ref,
        "roofline": roof,
        "roofline_near_field": roof_nf,
        "measured_rates": rates,
        "tree_build": {"ms": tree_ms, "points_per_s": N_POINTS / (tree_ms * 1e-3),
                       "note": "bin + sort + leaf offsets of 2^20 points (outside the timed evaluate)"},
        "speedup_mixed_vs_fp64": (results[f"fp64@{he:g}"]["ms_per_step"] / results[f"mixed@{he:g}"]["ms_per_step"]
                                  if "ms_per_step" in results.get(f"fp64@{he:g}", {})
                                  and "ms_per_step" in results.get(f"mixed@{he:g}", {}) else None),
        "cpu_baseline": cpu,
        "clocks": clocks,
        "variants": results,
        "workloads": workloads,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
