#!/usr/bin/env python3
"""Benchmark of randomized GENP on one GB300 (or N independent replicas).

One step = one pass of the whole method over one system, every step of it
in libgenp's kernels, called through the C ABI:
  a1 redraw the random multiplier G (new seed each step, no allocation)
  a2 C = A G
  a3-a5 blocked GENP of C (panel, TRSM, Schur update)
  a6-a7 L U y = B, X = G y
  a8 FP64 iterative refinement until the backward error is <= 1e-14
  a9 adjoint for the loss 0.5 ||X||_F^2 (gX = X): dA = -Lambda X^T, dB = Lambda
The default workload is the mixed-precision system: n = 16384,
A = J U diag(sigma) V^T with kappa(A) = 1e6, a dense Gaussian N(0, 1/n)
multiplier, one right-hand side, factors from BF16 tensor-core products by
exact digit slicing (7 digits) and GMRES-IR in FP64 to a backward error
<= 1e-14; the same system is then solved by the FP64 path on the same GPU
(1 warm-up + 1 timed step) for the comparison the metric names.  A, G and C
are 2 GiB each, larger than L2, so no flush is needed between steps.
`--workload lead --prec fp64 --n 8192 --nrhs 16` is the FP64 system at scale.

`--impl reference` times the CPU oracle (plain C, FP64) on a bounded sample
of the same workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & TFLOP/s (2n³/3), BF16+IR vs FP64 GENP, same GB300, bwd err ≤1e-14"
KINDS = {"gaussian": 0, "circulant": 1, "sparse": 2, "toeplitz": 5, "householder": 6}
PRECS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp8": 3, "bf16x3": 4, "sliced": 5}
# sliced: G drawn on the FP32 grid; fp8: on the FP8 grid (e4m3 times one power of two)
GRID_OF = {"fp64": 0, "fp32": 1, "bf16": 2, "fp8": 3, "bf16x3": 2, "sliced": 5}
F64_FACTORS = ("fp64", "sliced")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nrhs", type=int, default=1)
    p.add_argument("--kind", default="gaussian", choices=list(KINDS))
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--tol", type=float, default=1e-14)
    p.add_argument("--workload", default="svd",
                   choices=["lead", "svd", "batched", "diff", "small", "table71", "lowrank"],
                   help="lead: N(0,1) A with a rank-deficient leading block; svd: A = J U diag(sigma) V^T; "
                        "batched: 10k systems n in [16,512], a11 = 0, FP32 factors + FP64 refinement; "
                        "diff: 256 x n=1024 FP32 systems, circulant G, 8 RHS, forward + adjoint; "
                        "small: one n x n system of the lead recipe through the one-launch batched kernel; "
                        "table71: the paper-shaped Table 7.1 experiment (+-1 circulant multipliers, 100 systems "
                        "per n in 64, 256, 1024, residuals after 0 and 1 refinement steps, and plain GENP); "
                        "lowrank: the paper-shaped Tables 7.2 / 7.3 experiment (randomized rank-q approximation)")
    p.add_argument("--count", type=int, default=None, help="systems in the batched / diff workloads")
    p.add_argument("--kappa", type=float, default=1e6, help="condition number of the svd workload")
    p.add_argument("--prec", default="sliced", choices=list(PRECS))
    p.add_argument("--digits", type=int, default=0, help="digits per operand of the sliced precision (5, 6, 7)")
    p.add_argument("--precond-digits", type=int, default=None,
                   help="digits of A in the sliced C = A G (3 .. 7; 0: the library's setting, 7; default 5 with "
                        "GMRES-IR, which needs the product only as accurate as the factors it feeds)")
    p.add_argument("--mult-digits", type=int, default=0, choices=[0, 1, 2],
                   help="digits of the dense Gaussian multiplier's sliced grid (0: the library's setting, 1)")
    p.add_argument("--refine", default=None, choices=["classic", "gmres"],
                   help="refinement method (default: classic for fp64, GMRES-IR otherwise)")
    p.add_argument("--max-iter", type=int, default=None)
    p.add_argument("--nb", type=int, default=0, help="factorization block (0: the library's default)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-escalate", action="store_true",
                   help="batched: leave systems whose FP32 refinement stalls unconverged (no double-float refactor)")
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="skip timing the FP64 path on the same system (non-FP64 precisions)")
    p.add_argument("--no-configs", action="store_true",
                   help="default workload: skip the short measurements of the other configurations "
                        "(n = 256 and n = 8192 FP64, batched, differentiable) attached to the line")
    return p.parse_args()


def workload_name(a):
    prec = a.prec + (str(a.digits or 7) if a.prec == "sliced" else "")
    if a.workload == "svd":
        return f"genp_{prec}_n{a.n}_svd_kappa{a.kappa:.0e}_{a.kind}_{a.nrhs}rhs"
    return f"genp_{prec}_n{a.n}_{a.kind}_{a.nrhs}rhs"


def flops_per_solve(a):
    n = a.n
    fact = 2.0 * n**3 / 3.0
    if a.kind == "gaussian":
        ag = 2.0 * n**3
    elif a.kind == "circulant":
        ag = 2 * 5.0 * n * n * math.log2(n)      # forward + inverse complex FFT per row pair
    elif a.kind == "toeplitz":
        ag = 2 * 5.0 * n * (2 * n) * math.log2(2 * n)   # the same on the order-2n circulant embedding
    elif a.kind == "householder":
        ag = 4.0 * n * n                         # A u, then the rank-one update
    else:
        ag = 2.0 * 4 * n * n
    return fact, ag


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device) -> float:
    """The largest x over the ranks (every rank gets it): the job's time is
    its slowest replica's."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas: every rank solves its own systems)."""
    return world * units_per_rank / (ms / 1e3)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool):
        self.index, self.enabled, self.proc, self.path = index, enabled, None, None

    def __enter__(self):
        if self.enabled:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                              "--format=csv,noheader,nounits", "-lms", "200"],
                                             stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            except OSError:
                self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU)

def oracle_sample(a, n_sample: int, repeats: int):
    """The oracle's whole pipeline on an n_sample system of the same recipe;
    returns (seconds per solve, threads)."""
    import numpy as np

    import oracle
    import workloads as W
    if a.workload == "svd":
        A, _, B = W.svd_kappa(n_sample, a.kappa, a.nrhs, seed=a.seed)
    else:
        lead = max(2, 64 * n_sample // a.n)      # same recipe: leading block n/128, rank half of it
        A, _, B = W.lead_deficient(n_sample, lead, lead // 2, a.nrhs, seed=a.seed)
    A, B = A.numpy(), B.numpy()
    oracle.lib()
    times = []
    for r in range(repeats):
        t0 = time.perf_counter()
        M = oracle.multiplier(KINDS[a.kind], n_sample, seed=r + 1)
        res = oracle.solve(A, B, M, refine_steps=10, tol=a.tol)
        x = res["x"]
        oracle.adjoint(A, x, x)
        times.append(time.perf_counter() - t0)
    threads = len(os.sched_getaffinity(0))
    return statistics.median(times), threads, res["eta"][-1]


def library_gepp_sample(a, n_sample: int):
    """A library CPU reference beside the oracle: LAPACK's GEPP (scipy
    lu_factor / lu_solve, dgetrf / dgetrs, the host's BLAS threads) on an
    n_sample system of the same recipe, one refinement step in FP64; None
    when scipy is missing.  Returns (seconds per solve, backward error)."""
    try:
        import numpy as np
        import scipy.linalg as sla
    except ImportError:
        return None
    import workloads as W
    if a.workload == "svd":
        A, _, B = W.svd_kappa(n_sample, a.kappa, a.nrhs, seed=a.seed)
    else:
        lead = max(2, 64 * n_sample // a.n)
        A, _, B = W.lead_deficient(n_sample, lead, lead // 2, a.nrhs, seed=a.seed)
    A, B = A.numpy(), B.numpy()
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        lu = sla.lu_factor(A, check_finite=False)
        X = sla.lu_solve(lu, B, check_finite=False)
        X = X + sla.lu_solve(lu, B - A @ X, check_finite=False)
        times.append(time.perf_counter() - t0)
    R = B - A @ X
    eta = float(np.max(np.abs(R)) / (np.max(np.sum(np.abs(A), axis=1)) * np.max(np.abs(X)) + np.max(np.abs(B))))
    return statistics.median(times), eta


def oracle_batch_seconds(a, sizes, budget_s):
    """Oracle pipeline on the first systems of a batch for about budget_s;
    returns (seconds scaled to the whole batch by sum n^3, systems done)."""
    import oracle
    diff = a.workload == "diff"
    nrhs = 8 if diff else 4
    rng = np.random.default_rng(a.seed)
    t0, done = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and done < len(sizes):
        n = int(sizes[done])
        Ai = rng.standard_normal((n, n)) + (0.1 * n * np.eye(n) if diff else 0.0)
        if not diff:
            Ai[0, 0] = 0.0
        Bi = Ai @ rng.standard_normal((n, nrhs))
        res = oracle.solve(Ai, Bi, oracle.multiplier(1 if diff else 0, n, seed=done, grid="fp32"),
                           refine_steps=0 if diff else 10, tol=a.tol)
        if diff:
            oracle.adjoint(Ai, res["x"], res["x"])
        done += 1
    el = time.perf_counter() - t0
    frac = sum(float(n) ** 3 for n in sizes[:done]) / sum(float(n) ** 3 for n in sizes)
    return el / frac, done


def run_reference_batched(a):
    import workloads as W
    world, rank, _ = dist_env()
    if rank != 0:
        return
    diff = a.workload == "diff"
    count = a.count or (256 if diff else 10000)
    sizes = [1024] * count if diff else W.batched_sizes(count, 16, 512, seed=a.seed)
    per = []
    for i in range(a.warmup + a.steps):
        t, done = oracle_batch_seconds(a, sizes, 4.0)
        if i >= a.warmup:
            per.append(t)
    sec = statistics.mean(per)
    value = count / sec
    name = "batched_10k_n16-512_fp32_fp64ir_4rhs" if not diff else "diff_256x1024_fp32_circulant_8rhs"
    if small:
        name = f"onelaunch_n{a.n}_fp32_fp64ir_{nrhs}rhs"
    sample = f"oracle pipeline on the first {done} systems of the batch (~4 s per step), scaled by sum n^3"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "count": count},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(a):
    if a.workload in ("batched", "diff"):
        return run_reference_batched(a)
    world, rank, _ = dist_env()
    if rank != 0:
        return
    n_s = min(a.n, 2048)
    scale = (a.n / n_s) ** 3
    sec = []
    for i in range(a.warmup + a.steps):
        t, threads, eta = oracle_sample(a, n_s, 1)
        if i >= a.warmup:
            sec.append(t * scale)
    per = statistics.mean(sec)
    value = 1.0 / per
    sample = (f"oracle pipeline (multiplier, A G, GENP, solves, FP64 refinement, adjoint) on an n={n_s} system of "
              f"the same recipe, {a.nrhs} RHS; time scaled by (n/{n_s})^3 to n={a.n}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "n": a.n, "nrhs": a.nrhs, "multiplier": a.kind,
                       "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "bwd_err": eta}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours (GPU)

def run_ours(a, emit=True):
    import torch
    import torch.distributed as dist

    import paper_1212_4560_gb300 as genp
    import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1212_4560_gb300 import build as _b
    _b.build()

    n, nrhs = a.n, a.nrhs
    if a.workload == "svd":
        A, _, B = W.svd_kappa(n, a.kappa, nrhs, seed=a.seed + rank, device=dev)
        A_cpu, B_cpu = A.cpu(), B.cpu()
    else:
        lead = 32 if n <= 256 else 64          # n = 256: 32 x 32 of rank 16; larger n: 64 x 64 of rank 32
        A_cpu, _, B_cpu = W.lead_deficient(n, lead, lead // 2, nrhs, seed=a.seed + rank)
        A = A_cpu.to(dev)
        B = B_cpu.to(dev)
    prec = PRECS[a.prec]
    if a.digits:
        genp._lib.load().genp_sliced_digits(a.digits)
    method_name = a.refine or ("classic" if a.prec == "fp64" else "gmres")
    if a.precond_digits is None:
        a.precond_digits = 5 if (a.prec == "sliced" and method_name == "gmres") else 0
    old_pdigits = genp._lib.load().genp_sliced_precondition_digits(0)
    genp._lib.load().genp_sliced_precondition_digits(a.precond_digits or old_pdigits)
    if a.mult_digits:
        genp._lib.load().genp_sliced_multiplier_digits(a.mult_digits)
    cdt = torch.float64 if a.prec in F64_FACTORS else torch.float32
    method = {"classic": 0, "gmres": 1}[a.refine or ("classic" if a.prec == "fp64" else "gmres")]
    max_iter = a.max_iter if a.max_iter is not None else (10 if a.prec == "fp64" or method == 1 else 30)
    C = torch.empty((n, n), dtype=cdt, device=dev)
    X = torch.empty((n, nrhs), dtype=torch.float64, device=dev)
    dA = torch.empty((n, n), dtype=cdt, device=dev)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=dev)
    kind = KINDS[a.kind]
    G = genp.make_multiplier(kind, n, seed=1, stream_id=rank, value_grid=GRID_OF[a.prec])
    genp.precondition(G, A, C, c_prec=prec)
    F = genp.factor(C, prec=prec, nb=a.nb)
    stream = torch.cuda.current_stream(dev)

    def step(i, ev=None, Ain=None, Bin=None):
        Ai = A if Ain is None else Ain
        Bi = B if Bin is None else Bin

        def mark(k):
            if ev is not None:
                ev[k].record(stream)
        mark(0)
        genp.redraw_multiplier(G, seed=1000 + i, stream_id=rank)
        mark(1)
        genp.precondition(G, Ai, C, c_prec=prec)
        mark(2)
        genp.refactor(F, C)
        mark(3)
        genp.solve(F, G, Bi, X)
        mark(4)
        genp.refine(Ai, F, G, Bi, X, tol=a.tol, max_iter=max_iter, method=method)
        mark(5)
        genp.adjoint(F, G, X, X, dA, dB)
        mark(6)

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    info_w = genp.info_fetch(F)

    phases = ["multiplier", "precondition", "factor", "solve", "refine", "adjoint"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(a.steps)]
    lib = genp._lib.load()
    # CUDA events around every launch of the profiled kernel classes in the timed region
    lib.genp_profile_enable(1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = genp.launch_count()
    etas, iters = [], []
    with ClockSampler(local, not a.no_clocks and rank == 0) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(a.steps):
            step(a.warmup + i, evs[i])
        t_end.record(stream)
        torch.cuda.synchronize()
    launches = genp.launch_count() - l0
    tc_prof = None
    tc_launches = None
    class_prof = {}
    if True:
        import ctypes
        cnt = ctypes.c_int()
        lib.genp_profile_launches(None, None, 0, ctypes.byref(cnt))
        if cnt.value > 0:
            l_ms, l_fl = (ctypes.c_double * cnt.value)(), (ctypes.c_double * cnt.value)()
            lib.genp_profile_launches(l_ms, l_fl, cnt.value, ctypes.byref(cnt))
            tc_launches = (list(l_ms), list(l_fl))
        for cls in range(6):    # per kernel class: summed ms, algorithmic work, launches
            c_ms, c_w, c_n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
            if lib.genp_profile_class(cls, ctypes.byref(c_ms), ctypes.byref(c_w), ctypes.byref(c_n)) == 0:
                class_prof[cls] = (c_ms.value, c_w.value, c_n.value)
        p_ms, p_fl, p_n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        lib.genp_profile_read(ctypes.byref(p_ms), ctypes.byref(p_fl), ctypes.byref(p_n))
        lib.genp_profile_enable(0)
        tc_prof = (p_ms.value, p_fl.value, p_n.value)
    # the refinement runs as a cached CUDA graph in the timed steps, and the
    # launch profile skips what a graph holds: one more (untimed) step with
    # the refinement enqueued launch by launch gives the per-class rates
    info = genp.info_fetch(F)             # the last timed step's report
    eager_prof = {}
    if a.prec != "fp8":
        prev_graphs = lib.genp_refine_graphs(0)
        lib.genp_profile_enable(1)
        step(a.warmup + a.steps)
        torch.cuda.synchronize()
        import ctypes
        for cls in range(1, 6):
            c_ms, c_w, c_n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
            if lib.genp_profile_class(cls, ctypes.byref(c_ms), ctypes.byref(c_w), ctypes.byref(c_n)) == 0:
                eager_prof[cls] = (c_ms.value, c_w.value, c_n.value)
        lib.genp_profile_enable(0)
        lib.genp_refine_graphs(prev_graphs)
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    phase_ms = {p: sum(evs[i][k].elapsed_time(evs[i][k + 1]) for i in range(a.steps)) / a.steps
                for k, p in enumerate(phases)}
    total_ms = reduce_max(total_ms, world, dev)
    ms_per_step = total_ms / a.steps
    value = job_rate(world, a.steps, total_ms)
    fact, ag = flops_per_solve(a)
    tflops = world * (fact + ag) * a.steps / (total_ms / 1e3) / 1e12

    # e2e: the same step through the C ABI with the system in pinned HOST memory;
    # every step's copies in (A, B) and out (X) sit inside the timed region.
    # The inputs are double-buffered: step i + 1's A and B travel on a copy
    # stream while step i solves (a stream of systems, as a server sees it).
    e2e = None
    if not a.no_e2e:
        A_h = A_cpu.pin_memory()
        B_h = B_cpu.pin_memory()

        X_h = [torch.empty((n, nrhs), dtype=torch.float64).pin_memory() for _ in range(2)]
        Ab, Bb = [A, torch.empty_like(A)], [B, torch.empty_like(B)]
        cs = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        # the same multiplier seeds as the timed steps above, so that the two
        # figures differ only by the copies (the Krylov count varies by seed)
        k_e2e = a.steps

        def e2e_run(k, base):
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                Ab[0].copy_(A_h, non_blocking=True)
                Bb[0].copy_(B_h, non_blocking=True)
                copied[0].record(cs)
            for i in range(k):
                b = i % 2
                if i + 1 < k:
                    nb = (i + 1) % 2
                    with torch.cuda.stream(cs):
                        if i >= 1:
                            cs.wait_event(used[nb])
                        Ab[nb].copy_(A_h, non_blocking=True)
                        Bb[nb].copy_(B_h, non_blocking=True)
                        copied[nb].record(cs)
                stream.wait_event(copied[b])
                step(base + i, Ain=Ab[b], Bin=Bb[b])
                used[b].record(stream)
                X_h[b].copy_(X, non_blocking=True)

        e2e_run(2, 10_000)          # both input buffers once (their refinement graphs are recorded here)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_run(k_e2e, a.warmup)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        e_ms = reduce_max(e_ms, world, dev)
        e2e = {"value": job_rate(world, k_e2e, e_ms), "unit": "solves/s",
               "h2d_bytes_per_step": A_h.numel() * 8 + B_h.numel() * 8, "d2h_bytes_per_step": X_h[0].numel() * 8,
               "steps": k_e2e, "inputs": "double-buffered: step i+1's copy overlaps step i",
               "seeds": "the timed steps' multiplier seeds", "A_h_pinned": bool(A_h.is_pinned())}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # dominant kernel: the GEMM of C = A G (one launch per BF16 term / per FP64 call)
    peaks = measured_peaks()
    if a.prec == "sliced" and tc_prof and tc_prof[2] > 0:
        nd = lib.genp_sliced_digits(0)
        pd = lib.genp_sliced_precondition_digits(0)
        pairs = nd * (nd + 1) // 2
        t_ms, t_fl, t_n = tc_prof
        # the method's own work: each launch is an FP64-class product of 2 m n K
        # flop; the tensor pipe runs `pairs` digit products for each of them
        t_alg = class_prof[0][1] if 0 in class_prof else t_fl / pairs
        achieved = t_alg / (t_ms / 1e3) / 1e12
        pipe = t_fl / (t_ms / 1e3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        roofline = {"kernel": f"k_tc_sliced (tcgen05 BF16 digit products: A G and the Schur updates, FP64-class)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "measured bf16_tflops_sustained (kernel timed inside a long step)"
                    if "bf16_tflops_sustained" in peaks else "fallback",
                    "launches": t_n, "avg_launch_ms": t_ms / t_n,
                    "share_of_step": (t_ms / a.steps) / ms_per_step,
                    "algorithmic": "2 m n K flop per launch: the FP64-class product's own work (A G chunks, "
                                   "Schur updates)",
                    "tensor_pipe": {"achieved": pipe, "frac": pipe / peak, "unit": "TFLOP/s",
                                    "counted": "BF16 digit-pair products actually issued (2 m n Kpad per pair)"},
                    # dram read + write bytes of one n = 4096 A G chunk launch (K = 1024,
                    # column-major tile order) under ncu on the current kernel: 266.2 MB for
                    # k_tc_sliced<1, 5> (the one-digit multiplier grid), 281.7 MB for
                    # k_tc_sliced<2, 5> (two digits); the double-float accumulator's
                    # read-modify-write is 268 MB of either, the digit slices are read about
                    # once; scaled by the n^2 output tiles to this size's chunk launches
                    "traffic": (266.2e6 if lib.genp_sliced_multiplier_digits(0) == 1 else 281.7e6) * (n / 4096) ** 2
                    if (nd == 7 and pd == 5) else None,
                    "traffic_basis": "A G chunk launch (K = 1024) of k_tc_sliced<1 or 2, 5>; ncu at n = 4096 scaled "
                                     "by n^2; Schur-update launches (K = 512) read and write the same accumulator "
                                     "per tile over half the depth"}
    elif a.prec == "fp8" and tc_launches:
        # per launch: the A G product (K = n, k_tc_e4m3, tensor-bound) and the
        # Schur updates (K = nb <= 128, k_tc_gemm<true>, HBM-bound: C read and
        # written once, 8 B per entry); flops 2 m n K, so the update's m = n' is
        # sqrt(flops / (2 K)) with K = 128 (the last, ragged block aside)
        l_ms, l_fl = tc_launches
        ag = [(t, f) for t, f in zip(l_ms, l_fl) if f >= 2.0 * n**3 * 0.999]
        su = [(t, f) for t, f in zip(l_ms, l_fl) if f < 2.0 * n**3 * 0.999]
        base = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        fp8_peak = 2.0 * base
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        su_ms = sum(t for t, _ in su)
        su_bytes = sum(8.0 * (f / 256.0) for _, f in su)        # m^2 = f / (2 K), 8 B per C entry
        ag_ms = sum(t for t, _ in ag)
        ag_tf = sum(f for _, f in ag) / (ag_ms / 1e3) / 1e12 if ag_ms > 0 else None
        dominant_su = su_ms >= ag_ms
        if dominant_su:
            achieved = su_bytes / (su_ms / 1e3) / 1e9
            roofline = {"kernel": "k_tc_gemm<true> (tcgen05 kind::f8f6f4 Schur updates, K = 128: C22 read and written)",
                        "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "peak_source": "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback",
                        "launches": len(su), "avg_launch_ms": su_ms / len(su),
                        "share_of_step": (su_ms / a.steps) / ms_per_step,
                        "algorithmic": "8 B per C22 entry (FP32 read + write) per launch", "traffic": None}
        else:
            achieved = ag_tf
            roofline = {"kernel": "k_tc_e4m3 (tcgen05 kind::f8f6f4 C = A G, FP32 promotion per 128-wide k-tile)",
                        "bound": "tensor", "achieved": achieved, "peak": fp8_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp8_peak, "launches": len(ag), "avg_launch_ms": ag_ms / len(ag),
                        "share_of_step": (ag_ms / a.steps) / ms_per_step, "algorithmic": "2 n^3 e4m3 flop per launch",
                        "traffic": None}
        roofline["A_G_kernel"] = {"kernel": "k_tc_e4m3", "achieved_tflops": ag_tf, "peak": fp8_peak,
                                  "frac": (ag_tf / fp8_peak) if ag_tf else None, "avg_launch_ms":
                                  ag_ms / len(ag) if ag else None,
                                  "peak_source": "measured bf16_tflops_sustained x 2 (dense e4m3 / bf16 tensor "
                                                 "rate, 4.5 / 2.25 PFLOP/s nominal)"}
    elif a.kind == "gaussian" and a.prec in ("bf16", "bf16x3"):
        terms = 3 if a.prec == "bf16x3" else 1
        achieved = terms * 2.0 * n**3 / (phase_ms["precondition"] / 1e3) / 1e12
        peak = float(peaks.get("bf16_tflops", 1900.0))
        roofline = {"kernel": f"k_tc_gemm (tcgen05 BF16, C = A G, {terms} launch(es))", "bound": "tensor",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "measured bf16_tflops (burst)" if "bf16_tflops" in peaks else "fallback",
                    "traffic": None}
    elif a.kind == "gaussian" and a.prec == "fp32":
        achieved = 2.0 * n**3 / (phase_ms["precondition"] / 1e3) / 1e12
        peak = 152 * 128 * 2 * 2.070e9 / 1e12
        roofline = {"kernel": "k_gemm<float,128,128,8,8,8> (C = A G)", "bound": "alu", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz", "traffic": None}
    elif a.kind == "gaussian":
        achieved = 2.0 * n**3 / (phase_ms["precondition"] / 1e3) / 1e12
        roofline = {"kernel": "k_gemm<double,64,64,16,4,4> (C = A G)", "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 has no tensor-core path)",
                    # dram read+write bytes of one n=4096 launch under ncu (3.908e9), scaled by the
                    # flop count to the launch size timed here (both grow as n^3)
                    "traffic": 3.908e9 * (n / 4096) ** 3}
    else:
        achieved = (fact) / (phase_ms["factor"] / 1e3) / 1e12
        roofline = {"kernel": "GENP factor (Schur GEMM dominant)", "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz", "traffic": None}
    roofline["other_kernels"] = other_kernels(eager_prof or class_prof, 1 if eager_prof else a.steps, ms_per_step,
                                              peaks)
    if eager_prof:
        roofline["other_kernels_basis"] = ("one extra step after the timed ones with the refinement enqueued launch by "
                                           "launch (in the timed steps it runs as one cached CUDA graph)")
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        n_s = min(n, 2048)
        t, threads, _ = oracle_sample(a, n_s, 3)
        cpu = {"value": 1.0 / (t * (n / n_s) ** 3), "unit": "solves/s", "cores": threads, "kind": "oracle",
               "sample": f"oracle pipeline (multiplier, A G, GENP, solves, refinement, adjoint) on an n={n_s} "
                         f"system of the same recipe ({nrhs} RHS), median of 3, time scaled by (n/{n_s})^3 to n={n}"}
    cpu_lib = None
    if not a.no_cpu_baseline and world == 1:
        n_l = min(n, 4096)
        try:
            got = library_gepp_sample(a, n_l)
        except Exception:          # a context line only: never lose the bench line to it
            got = None
        if got is not None:
            t_l, eta_l = got
            cpu_lib = {"value": 1.0 / (t_l * (n / n_l) ** 3), "unit": "solves/s",
                       "cores": len(os.sched_getaffinity(0)), "kind": "LAPACK GEPP (scipy dgetrf/dgetrs)",
                       "bwd_err": eta_l,
                       "sample": f"GEPP + one FP64 refinement step on an n={n_l} system of the same recipe, "
                                 f"median of 3, time scaled by (n/{n_l})^3 to n={n}; a tuned library beside the "
                                 f"oracle, not the reference arm"}
    fp64 = None
    if a.prec != "fp64" and not a.no_fp64_compare and world == 1:
        fp64 = fp64_same_gpu(a, genp, A, B, kind, rank, dev)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "sliced": "bf16", "fp8": "e4m3"}.get(a.prec, a.prec),
            "data": "synthetic",
            "config": {"workload": workload_name(a), "n": n, "nrhs": nrhs, "multiplier": a.kind, "precision": a.prec,
                       "digits": {"factor": lib.genp_sliced_digits(0),
                                  "precondition": lib.genp_sliced_precondition_digits(0),
                                  "multiplier": lib.genp_sliced_multiplier_digits(0)}
                       if a.prec == "sliced" else None,
                       "A": ("J U diag(sigma) V^T, kappa=%g" % a.kappa) if a.workload == "svd"
                       else ("N(0,1) with leading 32x32 block of rank 16" if n <= 256
                             else "N(0,1) with leading 64x64 block of rank 32"),
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "bwd_err_unrefined": info.bwd_err[0] if info.bwd_err else None,
            "converged": bool(info.bwd_err) and info.bwd_err[-1] <= a.tol,
            "refine_method": ["classic", "gmres"][method],
            "tflops": tflops, "tflops_counted": {"factor_2n3_over_3": fact, "AG": ag},
            "phases_ms": phase_ms, "roofline": roofline, "cpu_baseline": cpu, "cpu_library": cpu_lib, "e2e": e2e,
            "gpu_launches": launches, "gpu_launches_per_step": launches / a.steps,
            "bwd_err": info.bwd_err[-1] if info.bwd_err else None, "refine_iters": info.refine_iters,
            "krylov_steps": info.krylov_steps,
            "breakdown_step": info.breakdown_step, "growth": info.growth, "status": info.status,
            "warmup_bwd_err": info_w.bwd_err[-1] if info_w.bwd_err else None}
    if fp64 is not None:
        line["fp64_same_gpu"] = fp64
        line["speedup_vs_fp64"] = value / fp64["value"] if fp64["value"] else None
    if not a.no_clocks:
        line["clocks"] = clk.summary()
    if not emit:
        return line
    if world == 1 and a.workload == "svd" and not a.no_configs:
        line["configs"] = other_configs(a)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def other_configs(a):
    """Short measurements of the other workloads, run after the headline one
    in the same process and attached to its line under "configs" (each its
    own CUDA-event timing, warm-up and oracle-free checks; no e2e or CPU legs)."""
    import copy
    base = copy.copy(a)
    base.no_e2e = base.no_cpu_baseline = base.no_clocks = base.no_fp64_compare = True
    base.digits = 0
    base.precond_digits = None
    base.refine = base.max_iter = None
    base.count = None
    runs = [("n256_fp64_gaussian_1rhs", run_ours, dict(workload="lead", n=256, nrhs=1, prec="fp64",
                                                         kind="gaussian", steps=50, warmup=5)),
            ("n256_onelaunch_fp32_fp64ir_1rhs", run_batched, dict(workload="small", n=256, nrhs=1, steps=50,
                                                                  warmup=5))]
    for kind in ("gaussian", "circulant", "sparse"):
        runs.append((f"n8192_fp64_{kind}_16rhs", run_ours, dict(workload="lead", n=8192, nrhs=16, prec="fp64",
                                                                 kind=kind, steps=2, warmup=1)))
    runs.append(("n8192_sliced_gaussian_16rhs", run_ours, dict(workload="lead", n=8192, nrhs=16, prec="sliced",
                                                               kind="gaussian", steps=3, warmup=2)))
    runs.append(("batched_10k_n16-512", run_batched, dict(workload="batched", steps=5, warmup=3)))
    runs.append(("diff_256x1024", run_batched, dict(workload="diff", steps=5, warmup=3)))
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "tflops", "roofline", "phases_ms",
            "bwd_err", "bwd_err_unrefined", "converged", "refine_iters", "gpu_launches_per_step", "bwd_err_max",
            "converged_fraction", "escalated_double_float", "growth")
    out = {}
    for name, fn, over in runs:
        b = copy.copy(base)
        for k, v in over.items():
            setattr(b, k, v)
        try:
            line = fn(b, emit=False)
            out[name] = {k: line[k] for k in keep if k in line}
        except Exception as exc:          # a side measurement never loses the headline line
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


PROF_CLASSES = {1: ("k_trsv", "streaming triangular solves; bytes = the factor's triangle, n^2/2 x 8 B per pass"),
                2: ("k_gemv", "x = G y, r = b - A x, the Krylov products A (G v); bytes = the matrix, n^2 x 8 B"),
                3: ("factor_aux", "factorization off the tensor cores: k_panel_reg, k_trsm_reg (double-float on "
                                  "the sliced path); flops of the diagonal blocks and block rows / columns"),
                4: ("k_outer", "adjoint dA = -Lambda X^T; bytes = dA written"),
                5: ("precondition_structured", "C = A G by the circulant FFT (k_circ_apply) or the sparse signed "
                                               "gather (k_sparse_pre); bytes = A read + C written, 16 n^2")}


def other_kernels(class_prof, steps, ms_per_step, peaks):
    """Achieved rate of each profiled kernel class (CUDA events around each
    launch in the timed region): HBM GB/s of algorithmic bytes against the
    measured copy rate, or flops for the factorization's latency-bound
    kernels."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    for cls, (name, what) in PROF_CLASSES.items():
        if cls not in class_prof or class_prof[cls][2] <= 0 or class_prof[cls][0] <= 0:
            continue
        ms_c, w_c, n_c = class_prof[cls]
        ent = {"launches": n_c, "ms_per_step": ms_c / steps, "share_of_step": (ms_c / steps) / ms_per_step,
               "counted": what}
        if cls == 3:
            ent.update(bound="latency", achieved=w_c / (ms_c / 1e3) / 1e12, unit="TFLOP/s")
        else:
            gbs = w_c / (ms_c / 1e3) / 1e9
            ent.update(bound="hbm", achieved=gbs, unit="GB/s", peak=hbm, frac=gbs / hbm,
                       peak_source="measured hbm_gbs" if "hbm_gbs" in peaks else "fallback")
        out[name] = ent
    return out


def fp64_same_gpu(a, genp, A, B, kind, rank, dev):
    """The FP64 path (FP64 product, FP64 GENP, classic FP64 refinement) on the
    same system and GPU: 1 warm-up step, then max(1, steps // 4) timed steps
    (each is about ten times a mixed-precision step)."""
    import torch
    n, nrhs = a.n, a.nrhs
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    X = torch.empty((n, nrhs), dtype=torch.float64, device=dev)
    dA = torch.empty((n, n), dtype=torch.float64, device=dev)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=dev)
    G = genp.make_multiplier(kind, n, seed=1, stream_id=rank, value_grid=genp.FP64)
    genp.precondition(G, A, C, c_prec=genp.FP64)
    F = genp.factor(C, prec=genp.FP64)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        genp.redraw_multiplier(G, seed=1000 + i, stream_id=rank)
        genp.precondition(G, A, C, c_prec=genp.FP64)
        genp.refactor(F, C)
        genp.solve(F, G, B, X)
        genp.refine(A, F, G, B, X, tol=a.tol, max_iter=10, method=0)
        genp.adjoint(F, G, X, X, dA, dB)

    step(a.warmup)
    torch.cuda.synchronize()
    k = max(1, a.steps // 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(k):
        step(a.warmup + 1 + i)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    info = genp.info_fetch(F)
    del F, G, C, X, dA, dB
    torch.cuda.empty_cache()
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "steps": k, "warmup": 1,
            "bwd_err": info.bwd_err[-1] if info.bwd_err else None, "refine_iters": info.refine_iters,
            "precision": "fp64 product, fp64 GENP, classic fp64 refinement"}


def run_batched(a, emit=True):
    """Many small systems per step: `batched` (uneven sizes, refinement) or
    `diff` (uniform n = 1024, forward + adjoint), one graph replay per step."""
    import torch
    import torch.distributed as dist

    import paper_1212_4560_gb300 as genp
    from paper_1212_4560_gb300 import batched as Bt
    import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1212_4560_gb300 import build as _b
    _b.build()
    diff = a.workload == "diff"
    small = a.workload == "small"
    if small:
        # one system through the one-launch batched kernel (count 1): the
        # n = 256 recipe, FP32 factors in one CTA, FP64 refinement
        count, nrhs = 1, a.nrhs
        sizes = [a.n]
        lead = 32 if a.n <= 256 else 64
        A1, _, B1 = W.lead_deficient(a.n, lead, lead // 2, nrhs, seed=a.seed + rank)
        plan = Bt.BatchedPlan(sizes, nrhs, kind=genp.GAUSSIAN, a_dtype=torch.float64,
                              max_iter=10 if a.max_iter is None else a.max_iter, tol=a.tol, escalate=True)
        Ap = A1.reshape(-1).to(dev).contiguous()
        Bp = B1.reshape(-1).to(dev).contiguous()
    elif diff:
        count = a.count or 256
        nrhs = 8
        sizes = [1024] * count
        A, _, Bm = W.shifted(count, 1024, nrhs, seed=a.seed + rank, device=dev, dtype=torch.float32)
        Ap = A.reshape(-1).contiguous()
        Bp = Bm.double().reshape(-1).contiguous()
        plan = Bt.BatchedPlan(sizes, nrhs, kind=genp.CIRCULANT, a_dtype=torch.float32, max_iter=10, tol=a.tol)
        del A
    else:
        count = a.count or 10000
        nrhs = 4
        sizes = W.batched_sizes(count, 16, 512, seed=a.seed + rank)
        plan = Bt.BatchedPlan(sizes, nrhs, kind=genp.GAUSSIAN, a_dtype=torch.float64,
                              max_iter=10 if a.max_iter is None else a.max_iter, tol=a.tol,
                              autotune=True, escalate=not a.no_escalate)
        Ap = torch.empty(plan.mat_size, dtype=torch.float64, device=dev)
        Bp = torch.empty(plan.vec_size, dtype=torch.float64, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(a.seed * 1_000_003 + 7919 + rank)
        for i, n in enumerate(sizes):
            Ai = torch.randn(n, n, generator=g, device=dev, dtype=torch.float64)
            Ai[0, 0] = 0.0
            Xi = torch.randn(n, nrhs, generator=g, device=dev, dtype=torch.float64)
            Ap[plan.mat_off[i]:plan.mat_off[i + 1]] = Ai.reshape(-1)
            Bp[plan.vec_off[i]:plan.vec_off[i + 1]] = (Ai @ Xi).reshape(-1)
    Xp = torch.empty_like(Bp)
    dA = torch.empty(plan.mat_size, dtype=torch.float32, device=dev) if diff else None
    dB = torch.empty_like(Bp) if diff else None
    stream = torch.cuda.current_stream(dev)

    def step_body(seed):
        plan.run(seed, Ap, Bp, Xp)
        if diff:
            plan.adjoint(Ap, Xp, Xp, dA, dB)    # loss 0.5 ||X||^2, refined like the forward

    # capture one step in a CUDA graph (allocation-free, no synchronization inside)
    s = torch.cuda.Stream(dev)
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        for i in range(max(1, a.warmup)):
            step_body(1 + i)
    stream.wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l_before = genp.launch_count()
    with torch.cuda.graph(graph):
        step_body(1)
    launches_per_step = genp.launch_count() - l_before
    for _ in range(a.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local, not a.no_clocks and rank == 0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    total_ms = reduce_max(e0.elapsed_time(e1), world, dev)
    st = plan.status()
    value = job_rate(world, count * a.steps, total_ms)
    n3 = sum(float(n) ** 3 for n in sizes)
    fact, ag = 2.0 * n3 / 3.0, (2.0 * n3 if not diff else sum(10.0 * n * n * np.log2(n) for n in sizes))
    tflops = world * (fact + ag) * a.steps / (total_ms / 1e3) / 1e12
    peak = 152 * 128 * 2 * 2.070e9 / 1e12
    # The FP64 residuals r = b - A x of the refinement (2 n^2 nrhs flop per
    # outer step and system) run on units 64 times slower than the FP32 pipe:
    # counted as 64 FP32-equivalent flop each in the ALU roofline below.
    iters = np.asarray(st["iters"], dtype=np.float64)
    fp64_flop = float(sum(2.0 * float(nn) ** 2 * nrhs * (it + 1) for nn, it in zip(sizes, iters)))
    eq_tflops = world * (fact + ag + 64.0 * fp64_flop) * a.steps / (total_ms / 1e3) / 1e12
    e2e = None
    if not a.no_e2e:
        A_h = Ap.cpu().pin_memory()
        B_h = Bp.cpu().pin_memory()
        X_h = torch.empty(Xp.shape, dtype=Xp.dtype).pin_memory()
        k = max(2, min(a.steps, 4))
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(k):
            Ap.copy_(A_h, non_blocking=True)
            Bp.copy_(B_h, non_blocking=True)
            graph.replay()
            X_h.copy_(Xp, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": job_rate(world, count * k, reduce_max(f0.elapsed_time(f1), world, dev)), "unit": "solves/s",
               "h2d_bytes_per_step": A_h.numel() * A_h.element_size() + B_h.numel() * 8,
               "d2h_bytes_per_step": X_h.numel() * 8, "steps": k}
    # one more (eager, untimed) run with the kernel's phase profile on: SM
    # cycles by phase, summed over the persistent CTAs
    plan.profile(True)
    step_body(1)
    phases = plan.profile_read()
    plan.profile(False)
    tot = sum(phases.values()) or 1.0
    phase_share = {k: round(v / tot, 4) for k, v in phases.items()}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if not a.no_cpu_baseline and world == 1 and not small:
        t, done = oracle_batch_seconds(a, sizes, 15.0)
        cpu = {"value": count / t, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"oracle pipeline on the first {done} systems of the batch (~15 s), scaled to the "
                         f"whole batch by sum n^3"}
    name = "batched_10k_n16-512_fp32_fp64ir_4rhs" if not diff else "diff_256x1024_fp32_circulant_8rhs"
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "count": count, "nrhs": nrhs,
                       "sizes": (str(a.n) if small else ("uniform [16, 512]" if not diff else "1024")),
                       "multiplier": "gaussian" if not diff else "circulant",
                       "precision": "fp32 factors" + (", fp64 refinement" if not diff else ", forward + adjoint"),
                       "l2": "inputs larger than L2 (no flush)", "graph": "one CUDA graph replay per step",
                       "block_sizes": {str(nn): plan.block_size(nn) for nn in (16, 128, 512, 1024)}},
            "tflops": tflops,
            "roofline": {"kernel": "k_batched (persistent: CTA-level FFMA GEMM, FP64 residuals)", "bound": "alu",
                         "achieved": eq_tflops / world, "peak": peak, "unit": "TFLOP/s (FP32-equivalent)",
                         "frac": eq_tflops / world / peak,
                         "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz",
                         "algorithmic": "(2/3 + 2) n^3 FP32 flop per system (factor + A G; 10 n^2 log2 n for the "
                                        "circulant A G) + 64 x the FP64 residual flop 2 n^2 nrhs (iters + 1) "
                                        "(GB300's FP64:FP32 throughput ratio); the double-float refactorization "
                                        "of escalated systems is not counted",
                         "fp32_only_frac": tflops / world / peak, "traffic": None},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * a.steps,
            "gpu_launches_per_step": launches_per_step,
            "bwd_err_max": float(np.max(st["eta"])), "bwd_err_unrefined_median": float(np.median(st["eta0"])),
            "converged_fraction": float(np.mean(st["eta"] <= a.tol)) if not diff else None,
            "refine_iters_mean": float(np.mean(st["iters"])),
            "fallback_substitution": int(np.sum(st["escalated"] == 1)),
            "escalated_double_float": int(np.sum(st["escalated"] == 2)),
            "krylov_steps_mean": float(np.mean(st["krylov"])),
            "phase_share_of_cta_cycles": phase_share}
    if not a.no_clocks:
        line["clocks"] = clk.summary()
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_table71(a):
    """Sec. 7.1 / Table 7.1, paper-shaped: for n = 64, 256, 1024 and 100 seeded
    systems each (workloads.table71: well conditioned, numerically singular
    n/2 x n/2 leading block), GENP of A G with the paper's circulant +-1
    multiplier, relative residual ||A y - b||_2 / ||b||_2 after 0 and 1 FP64
    refinement steps, and plain GENP (G = I) for comparison.  Statistics only:
    the paper does not give its matrices, so its numbers are context."""
    import torch

    import paper_1212_4560_gb300 as genp
    import workloads as W
    world, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1212_4560_gb300 import build as _b
    _b.build()
    count = a.count or 100

    def relres(A, X, B):
        return float(torch.linalg.norm(A @ X - B) / torch.linalg.norm(B))

    def stats(v):
        v = np.array(v)
        return {"min": float(v.min()), "max": float(v.max()), "mean": float(v.mean()), "std": float(v.std())}

    rows, plain = [], {}
    t0 = time.perf_counter()
    for n in (64, 256, 1024):
        r0, r1, rp, attempts = [], [], [], []
        for seed in range(count):
            A, _, B = W.table71(n, seed, device=dev)
            G = genp.make_multiplier(genp.CIRCULANT_PM1, n, seed=seed)
            C = torch.empty_like(A)
            genp.precondition(G, A, C)
            F = genp.factor(C)
            X = torch.empty_like(B)
            genp.solve(F, G, B, X)
            r0.append(relres(A, X, B))
            genp.refine(A, F, G, B, X, tol=0.0, max_iter=1)
            r1.append(relres(A, X, B))
            Gi = genp.make_multiplier(genp.IDENTITY, n, seed=0)
            Ci = A.clone()
            Fi = genp.factor(Ci)
            Xi = torch.empty_like(B)
            genp.solve(Fi, Gi, B, Xi)
            rp.append(relres(A, Xi, B))
        rows.append(dict(n=n, iterations=0, **stats(r0)))
        rows.append(dict(n=n, iterations=1, **stats(r1)))
        plain[str(n)] = stats([x if math.isfinite(x) else float("inf") for x in rp])
    line = {"workload": "table71_paper_shaped", "systems_per_n": count,
            "multiplier": "circulant, +-1 first column, redrawn on a zero DFT bin of power-of-two order",
            "residual": "||A y - b||_2 / ||b||_2", "rows": rows, "plain_genp": plain,
            "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_lowrank(a):
    """Sec. 7.2 / Tables 7.2 and 7.3, paper-shaped: for n = 64, 128, 256 and
    numerical rank q = 1, 8, 32 (workloads.lowrank: s_j = 1/j up to q,
    1e-10 beyond), 100 seeded matrices each, genp_lowrank with a Gaussian
    (Table 7.2) or Gaussian Toeplitz (Table 7.3, q = 8, 32) sketch of r = q
    columns; statistics of rn1 = ||B Y - T_q|| and rn2 = ||A - A Q Q^T||
    (2-norms, on the host).  The paper's inputs came from error-free ring
    operations on matrices it does not give: its numbers are context."""
    import torch

    import paper_1212_4560_gb300 as genp
    import workloads as W
    world, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1212_4560_gb300 import build as _b
    _b.build()
    count = a.count or 100

    def stats(v):
        v = np.array(v)
        return {"min": float(v.min()), "max": float(v.max()), "mean": float(v.mean()), "std": float(v.std())}

    rows = []
    t0 = time.perf_counter()
    gpu_ms = 0.0
    for toep in (False, True):
        for q in (1, 8, 32):
            if toep and q == 1:
                continue
            for n in (64, 128, 256):
                r1, r2 = [], []
                for seed in range(count):
                    A, S, T, s = W.lowrank(n, q, seed)
                    Ad = A.to(dev)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    G, Q, R, AQ, st = genp.lowrank(Ad, q, kind=genp.TOEPLITZ if toep else genp.GAUSSIAN, seed=seed)
                    e1.record()
                    torch.cuda.synchronize()
                    gpu_ms += e0.elapsed_time(e1)
                    An, Gn, Qn, AQn, Tn = (x.cpu().numpy() for x in (A, G, Q, AQ, T))
                    B = An.T @ Gn
                    Y = np.linalg.lstsq(B, Tn[:, :q], rcond=None)[0]
                    r1.append(float(np.linalg.norm(B @ Y - Tn[:, :q], 2)))
                    r2.append(float(np.linalg.norm(An - AQn @ Qn.T, 2)))
                rows.append(dict(sketch="toeplitz" if toep else "gaussian", q=q, n=n, rn1=stats(r1), rn2=stats(r2)))
    line = {"workload": "lowrank_tables_7_2_7_3_paper_shaped", "matrices_per_case": count, "rows": rows,
            "gpu_ms_total": gpu_ms, "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.workload == "table71":
        run_table71(a)
    elif a.workload == "lowrank":
        run_lowrank(a)
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload in ("batched", "diff", "small"):
        run_batched(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
