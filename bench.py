#!/usr/bin/env python
"""HODLR factor + solve benchmark on GB300 (one JSON line on stdout).

Step = one pass of the whole hot path on one batch of synthetic input:
low-precision factorization (leaf LU, leaf solves, per-level projections,
FP64 coupling matrices, ancestor updates), the solve recovered to an FP64
relative residual <= 1e-10 (FGMRES or iterative refinement, FP64 residual
matvec), and the log-determinant. The plain FP64 factor + solve is timed
beside it on the same inputs.

value = algorithmic factor + solve flops (the exact loop count of the FP64
algorithm, counted by paper_2208_06290_gb300.costs) / seconds per step,
whole job (N replicas under torchrun: one independent problem per GPU).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                       [--impl native|reference]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HODLR factor+solve seconds & TFLOP/s at N=2^20, mixed vs FP64, resid ≤1e-10"

# Workloads (shapes of the benchmark configurations). data: how the operator
# is generated (untimed).
WORKLOADS = {
    "bie-2^20": dict(N=1 << 20, L=13, r=32, k=1, prec="bf16", solver="gmres", shift=4.0, seed=2,
                     data="bie", desc="2D Laplace second-kind BIE on the star curve, N=2^20, leaf 128, rank 32, "
                                      "1 RHS; BF16-panel factor as FGMRES preconditioner to relres 1e-10"),
    "bie-2^17": dict(N=1 << 17, L=10, r=32, k=1, prec="bf16", solver="gmres", shift=4.0, seed=2,
                     data="bie", desc="2D Laplace BIE on the star curve, N=2^17, leaf 128, rank 32, 1 RHS (small "
                                      "case of the same structure, for profiler captures)"),
    "synthetic-4096": dict(N=4096, L=6, r=16, k=1, prec="fp64", solver="direct", shift=4.0, seed=0,
                           data="synthetic", desc="synthetic HODLR N=4096, leaf 64, rank 16, FP64"),
    "gaussian-2^18": dict(N=1 << 18, L=10, r=64, k=16, prec="fp32", solver="refine", restart=30, shift=0.0, seed=1,
                          data="gaussian", desc="Gaussian kernel (sigma 0.1, nugget 1e-2) on 2^18 kd-ordered points "
                                                "in [0,1]^2, leaf 256, rank 64, 16 RHS; FP32 factor + refinement, "
                                                "FGMRES(30) when refinement stalls"),
    "matern-2^20": dict(N=1 << 20, L=12, r=64, k=32, prec="fp32", solver="refine", restart=30, shift=0.0, seed=3,
                        grad=True,
                        data="matern", desc="Matern-3/2 kernel (lengthscale 0.2, nugget 1e-3) on 2^20 kd-ordered "
                                            "points in [0,1]^3, leaf 256, rank 64, 32 RHS; FP32 factor + refinement, "
                                            "FGMRES(30) when refinement stalls"),
    "synthetic-2^23": dict(N=1 << 23, L=15, r=32, k=64, prec="bf16", solver="refine", shift=8.0, seed=4,
                           data="synthetic", desc="synthetic HODLR N=2^23, leaf 256, rank 32, 64 RHS; BF16 "
                                                  "factor + refinement to 1e-10"),
}
DEFAULT_WORKLOAD = "bie-2^20"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ALU peaks for kernels bound by plain arithmetic, from the unit counts and the
# sampled SM clock: FP64 FMA pipe 2 FMA/clk/SM (4 flop), FP32 128 FMA/clk/SM
# (256 flop), 152 SMs.
FP64_FLOP_PER_CLK_PER_SM = 4.0
FP32_FLOP_PER_CLK_PER_SM = 256.0


def fp64_peak_tflops(sm_mhz):
    return 152 * FP64_FLOP_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz):
    return 152 * FP32_FLOP_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12


# DRAM traffic / algorithmic bytes of each kernel class, from one ncu capture
# of the current kernels at BIE N = 2^17 (DRAM read + write over the
# launcher's algorithmic bytes). The bench scales its per-launch algorithmic bytes by this ratio for
# `roofline.traffic` (the traffic of these kernels grows in proportion to the
# units processed). A class whose kernel changes loses its entry until it is
# captured again.
TRAFFIC_RATIO = {
    "matvec": 812.6 / 808.5,      # mv1_leaf_project_g8 + mv1_run_sum + mv1_node_sum + mv1_leaf_apply, one matvec
    "leaf_lu": 259.6 / 268.4,     # leaf_inv_tc_kernel
    "project_tc": 550.3 / 615.5,  # project_tc_kernel, the ten levels of one factorization
}
# (update_coupled_tc_kernel is left out: at N = 2^17 most of Y stays in L2,
# so the small case's ratio does not scale.)


def class_bound(cls, prec, m=128):
    """Resource that bounds each kernel class of the library's profiler:
    'hbm' (bytes), 'alu64' / 'alu32' (flops on the FP64 / FP32 pipes)."""
    if cls in ("vector", "reduce_chunks", "logdet"):
        return "hbm"
    if cls in ("matvec", "leaf_matvec"):
        return "alu64"          # FP64 residual matvec: 0.25 flop/B > FP64 ridge ~0.17 flop/B
    if prec == "fp64":
        return "alu64"
    if cls == "coupling":
        return "alu64"
    if cls == "leaf_lu":
        # leaves of 65..128 rows: blocked Gauss-Jordan with tensor-core updates
        return "hbm" if 64 < m <= 128 else "alu32"
    if prec == "fp32" and cls in ("leaf_solve", "project", "update", "coupling_apply"):
        return "alu32"
    return "hbm"


# ----------------------------------------------------------------- inputs
def reduced(w, log2_cap):
    """The workload with N reduced to at most 2^log2_cap (same leaf, rank,
    right-hand sides, operator family and seed): the bounded sample the CPU
    oracle is timed on."""
    N = min(w["N"], 1 << log2_cap)
    m = w["N"] >> w["L"]
    out = dict(w)
    out["N"], out["L"] = N, max(1, int(round(math.log2(N // m))))
    return out


def make_inputs(w, device, rank=0, stats=None):
    import torch
    from synth import HodlrShape, gaussian_rhs, synthetic_hodlr
    shape = HodlrShape(w["N"], w["L"], w["r"])
    if w["data"] in ("bie", "gaussian", "matern"):
        from synth.kernels import bie_hodlr, kernel_hodlr
        if w["data"] == "bie":
            D, U, V = bie_hodlr(shape, device=device, seed=w["seed"], stats=stats)
        elif w["data"] == "gaussian":
            D, U, V, pts = kernel_hodlr(shape, 2, "gaussian", 0.1, 1e-2, device=device, seed=w["seed"], stats=stats)
        else:
            D, U, V, pts = kernel_hodlr(shape, 3, "matern32", 0.2, 1e-3, device=device, seed=w["seed"], stats=stats)
        if stats is not None and w["data"] != "bie":
            stats["points"] = pts
        g = torch.Generator(device=device)
        g.manual_seed(w["seed"] + 1000 * rank)
    else:
        D, U, V, g = synthetic_hodlr(shape, w["shift"], w["seed"] + 1000 * rank, device=device)
    B = gaussian_rhs(w["N"], w["k"], g, device=device)
    return D, U, V, B


def cpu_model():
    """Host CPU model as the kernel reports it (x86 'model name'; on Arm the
    implementer/part pair when lscpu is absent)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "CPU part"):
            for line in info.splitlines():
                if line.startswith(key):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------- replicas (N > 1)
def max_over_ranks(x, world, device):
    """The largest per-rank value over the job (the rank's own when alone):
    the slowest replica sets the job's time."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_rank, world, seconds):
    """Whole-job throughput of `world` independent replicas, each doing
    flops_per_rank in the slowest rank's `seconds`."""
    return world * flops_per_rank / seconds / 1e12


# ----------------------------------------------------------------- clocks
CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
THROTTLE_NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def parse_clock_samples(lines, t0=None, t1=None):
    """Summarise nvidia-smi CSV lines (CLOCK_FIELDS, noheader, nounits): the
    median SM clock, the max clock and the active throttle reasons of the
    samples whose timestamp lies in [t0, t1] (epoch seconds, local time as
    nvidia-smi prints it); all samples if none does or no window is given."""
    import datetime
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            sm, smax = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None  # kept, but cannot be placed in the region
        rows.append((ts, sm, smax, parts[6:10]))
    inside = [x for x in rows if t0 is not None and t1 is not None and x[0] is not None and t0 <= x[0] <= t1]
    use = inside if inside else rows
    reasons = sorted({n for x in use for n, v in zip(THROTTLE_NAMES, x[3]) if v.lower().startswith("active")})
    return {"sm_mhz": statistics.median(x[1] for x in use) if use else None,
            "sm_max_mhz": max(x[2] for x in use) if use else None,
            "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


class ClockSampler:
    """nvidia-smi sampling every 50 ms in the background; start() returns once
    the first sample is written, so that the timed region is covered."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        deadline = time.time() + 5.0
        while time.time() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self, t0=None, t1=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_samples(f.readlines(), t0, t1)
        os.unlink(self.path)
        return out


# ----------------------------------------------------------------- native arm
def run_native(args, w, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2208_06290_gb300 import binding as hb
    from paper_2208_06290_gb300 import costs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    hb.hodlr_coupling_fp64_enable(args.coupling_fp64)
    N, L, r, k = w["N"], w["L"], w["r"], w["k"]
    m = N >> L
    gen_stats = {}
    D, U, V, B = make_inputs(w, dev, rank, stats=gen_stats)
    X = torch.empty(k, N, dtype=torch.float64, device=dev).T
    flops = costs.factor_flops(N, m, r, L) + costs.solve_flops(N, m, r, L, k)
    prec = w["prec"]
    stream = torch.cuda.current_stream()

    def step():
        F = hb.hodlr_factor(D, U, V, L, r, prec)
        if w["solver"] == "gmres":
            _, it, rr, code = hb.hodlr_gmres(F, D, U, V, B, tol=1e-10, restart=30, max_iter=args.gmres_max_iter,
                                             X=X, raise_on_fail=False)
        elif w["solver"] == "refine":
            _, it, rr, code = hb.hodlr_solve_refined(F, D, U, V, B, tol=1e-10, max_iter=50, X=X,
                                                     raise_on_fail=False, restart=w.get("restart", 0),
                                                     gmres_max_iter=args.gmres_max_iter)
        else:
            X.copy_(B)
            hb.hodlr_solve(F, X)
            it, rr, code = 0, None, 0
        sign, ld = hb.hodlr_logdet(F)
        return it, rr, code, sign, ld

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    # timed region: library profiler off (no per-launch events inside)
    sampler = ClockSampler(dev.index)
    sampler.start()
    launches0 = hb.hodlr_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    wall0 = time.time()
    e0.record(stream)
    info = [step() for _ in range(args.steps)]
    e1.record(stream)
    barrier()
    wall1 = time.time()
    launches = hb.hodlr_launch_count() - launches0
    clocks = sampler.stop(wall0, wall1)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    sec_step = ms_max / 1e3 / args.steps
    iters = [i[0] for i in info]
    relres = [i[1] for i in info]
    sign_mixed, ld_mixed = info[-1][3], info[-1][4]
    x_mixed = X.clone()
    # relres measured independently of the solver's own report
    res = hb.hodlr_matvec(D, U, V, L, r, X)
    res.sub_(B).neg_()
    rel_true = float((res.norm(dim=0) / B.norm(dim=0)).max().item())

    # per-kernel-class times: a separate pass of the same steps with the
    # library's per-launch CUDA-event brackets on (launching stream)
    nprof = max(1, min(args.steps, 5))
    hb.hodlr_profile_reset()
    hb.hodlr_profile_enable(True)
    for _ in range(nprof):
        step()
    hb.hodlr_profile_enable(False)
    prof = hb.hodlr_profile_read()
    work = hb.hodlr_profile_work()

    # plain FP64 factor + solve on the same inputs
    fp64 = None
    err_vs_fp64 = {}
    if not args.no_fp64:
        Xf = torch.empty_like(X)
        ld64 = [None, None]

        def step64():
            F64 = hb.hodlr_factor(D, U, V, L, r, "fp64")
            Xf.copy_(B)
            hb.hodlr_solve(F64, Xf)
            ld64[0], ld64[1] = hb.hodlr_logdet(F64)

        step64()
        barrier()
        n64 = max(1, min(args.steps, 2))
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n64):
            step64()
        a1.record(stream)
        barrier()
        s64 = a0.elapsed_time(a1) / 1e3 / n64
        r64 = hb.hodlr_matvec(D, U, V, L, r, Xf)
        r64.sub_(B).neg_()
        fp64 = {"seconds": s64, "tflops": flops / s64 / 1e12,
                "relres": float((r64.norm(dim=0) / B.norm(dim=0)).max().item()),
                "logdet": ld64[1], "sign": ld64[0],
                "speedup_of_mixed": s64 / sec_step}
        dx = (x_mixed - Xf)
        err_vs_fp64 = {
            "x_rel_err_vs_fp64": float((dx.norm(dim=0) / Xf.norm(dim=0)).max().item()),
            "x_max_abs_err_vs_fp64_over_max_abs": float((dx.abs().max() / Xf.abs().max()).item()),
            "logdet_mixed": ld_mixed, "logdet_fp64": ld64[1],
            "logdet_rel_err_vs_fp64": abs(ld_mixed - ld64[1]) / max(abs(ld64[1]), 1e-300),
            "sign_matches_fp64": sign_mixed == ld64[0],
        }

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        Dh, Uh, Vh, Bh = (tt.cpu().pin_memory() for tt in (D, U, V, B))
        Xh = torch.empty(k, N, dtype=torch.float64).pin_memory().T
        h2d = sum(tt.numel() * 8 for tt in (Dh, Uh, Vh, Bh))
        d2h = Xh.numel() * 8
        n_e2e = max(1, min(args.steps, 3))
        barrier()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(n_e2e):
            D.copy_(Dh, non_blocking=True)
            U.copy_(Uh, non_blocking=True)
            V.copy_(Vh, non_blocking=True)
            B.copy_(Bh, non_blocking=True)
            step()
            Xh.copy_(X, non_blocking=True)
        c1.record(stream)
        barrier()
        s_e2e = c0.elapsed_time(c1) / 1e3 / n_e2e
        s_e2e_max = max_over_ranks(s_e2e, world, dev)
        e2e = {"value": job_tflops(flops, world, s_e2e_max), "unit": "TFLOP/s", "seconds": s_e2e_max,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # adjoint solve B <- A^{-T} B with a factor of the step's precision, timed alone
    def timed(fn, n):
        fn()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(n):
            fn()
        t1.record(stream)
        barrier()
        return t0.elapsed_time(t1) / 1e3 / n

    Fa = hb.hodlr_factor(D, U, V, L, r, prec)
    Xa = torch.empty_like(X)

    def adj():
        Xa.copy_(B)
        hb.hodlr_solve_adjoint(Fa, Xa)

    adjoint = {"seconds": timed(adj, 3), "rhs": k, "factor_precision": prec,
               "bytes_per_solve_min": costs.solve_bytes(N, m, r, L, k, prec)}
    adjoint["achieved_gbs"] = adjoint["bytes_per_solve_min"] / adjoint["seconds"] / 1e9
    del Fa, Xa
    grad = None
    if w.get("grad") and not args.no_fp64:
        # backward of loss = sum b^T A^{-1} b + log|det A| (hodlr_grad) on an FP32
        # factor, and its error against the FP64 factor's gradient (untimed)
        F32 = hb.hodlr_factor(D, U, V, L, r, "fp32")
        g32 = [None]

        def back32():
            g32[0] = hb.hodlr_grad(F32, U, V, B, want_loss=False)

        t_grad = timed(back32, 2)
        del F32
        F64 = hb.hodlr_factor(D, U, V, L, r, "fp64")
        g64 = hb.hodlr_grad(F64, U, V, B, want_loss=False)
        del F64
        names = ("dD", "dU", "dV", "dB")
        grad = {"seconds": t_grad, "factor_precision": "fp32", "rhs": k,
                "rel_err_vs_fp64": {n: float(((a - b).norm() / b.norm()).item())
                                    for n, a, b in zip(names, g32[0][1:], g64[1:])}}
        del g32, g64
        torch.cuda.empty_cache()

    # the relative residual any FP64 solver can be expected to reach on this
    # operator: about eps |A|_2 |x| / |b| (backward-stable arithmetic); |A|_2
    # by power iteration on A (symmetric kernels) or A^T A (the BIE, with the
    # transposed operator D_b^T, U <-> V)
    def norm2_estimate(iters=20):
        sym = w["data"] in ("gaussian", "matern")
        Dt = None
        if not sym:  # D_b^T in the column-major block layout
            Dt = torch.empty_like(D.transpose(1, 2).contiguous()).transpose(1, 2)
            Dt.copy_(D.transpose(1, 2))
        g = torch.Generator(device=dev).manual_seed(11)
        v = torch.randn(1, N, generator=g, device=dev, dtype=torch.float64).T
        lam = 0.0
        for _ in range(iters):
            v = v / v.norm()
            y = hb.hodlr_matvec(D, U, V, L, r, v)
            if sym:
                lam = float(y.norm().item())
            else:
                y = hb.hodlr_matvec(Dt, V, U, L, r, y)
                lam = math.sqrt(float(y.norm().item()))
            v = y
        return lam

    normA = norm2_estimate()
    xn = float((X.norm(dim=0) / B.norm(dim=0)).max().item())
    attainable = {"norm2_A_estimate": normA, "max_x_over_b": xn,
                  "eps_normA_x_over_b": 1.1102230246251565e-16 * normA * xn}

    # GPU construction of the same operator family (hodlr_compress: exact leaf
    # blocks, partial-pivoted cross approximation at rank r), timed alone
    construction = None
    if w["data"] in ("bie", "gaussian", "matern"):
        kind = {"bie": "bie_star", "gaussian": "gaussian", "matern": "matern32"}[w["data"]]
        ckw = {"gaussian": dict(scale=0.1, nugget=1e-2), "matern": dict(scale=0.2, nugget=1e-3)}.get(w["data"], {})
        pts = gen_stats.get("points")

        def build_op():
            return hb.hodlr_compress(N, L, r, kind, pts, **ckw)

        t_c = timed(lambda: build_op(), 2)
        Dc, Uc, Vc = build_op()
        # relative difference from the randomized-SVD operator the step factors
        # (both approximate the same dense matrix; sampled rows, FP64 matvec)
        probe = torch.randn(1, N, generator=torch.Generator(device=dev).manual_seed(9), device=dev,
                            dtype=torch.float64).T
        y_c = hb.hodlr_matvec(Dc, Uc, Vc, L, r, probe)
        y_g = hb.hodlr_matvec(D, U, V, L, r, probe)
        construction = {"seconds": t_c, "kernel": kind, "rank": r, "method": "partial-pivoted cross approximation",
                        "rel_diff_vs_rsvd_operator_on_random_vector": float(((y_c - y_g).norm() / y_g.norm()).item())}
        del Dc, Uc, Vc, y_c, y_g
        torch.cuda.empty_cache()

    # FP64 pipe rate of this GPU, measured by the library's register-only
    # FMA probe (CUDA events on the launching stream, best of three)
    pk = peaks()
    sm_mhz = clocks.get("sm_mhz") or 1920.0
    fp64_meas = measure_fp64_tflops(hb, dev, stream)

    # roofline of every kernel class, from the profiled pass's CUDA-event
    # brackets; the line's roofline is the dominant (longest) class
    def roof_of(cls):
        cms, cn = prof[cls]
        cbytes, cflops = work[cls]
        bound = class_bound(cls, prec, m)
        if bound == "hbm":
            ach, peak, unit = cbytes / (cms / 1e3) / 1e9, pk["hbm_gbs"], "GB/s"
            src = f"MEASURED_PEAKS.json hbm_gbs ({pk['source']})"
        elif bound == "alu64":
            ach, unit = cflops / (cms / 1e3) / 1e12, "TFLOP/s"
            peak = fp64_meas["tflops"]
            src = (f"measured FP64 FMA probe: {fp64_meas['fmas']:.3e} FMA in {fp64_meas['ms']:.3f} ms "
                   f"(nominal {FP64_FLOP_PER_CLK_PER_SM:g} flop/clk/SM x 152 SMs x {sm_mhz:.0f} MHz = "
                   f"{fp64_peak_tflops(sm_mhz):.4f} TFLOP/s)")
        else:
            ach, unit = cflops / (cms / 1e3) / 1e12, "TFLOP/s"
            peak = fp32_peak_tflops(sm_mhz)
            src = f"FP32 pipe {FP32_FLOP_PER_CLK_PER_SM:g} flop/clk/SM x 152 SMs x median {sm_mhz:.0f} MHz"
        traffic = TRAFFIC_RATIO[cls] * cbytes / max(cn, 1) if cls in TRAFFIC_RATIO and prec == "bf16" else None
        return {"bound": "hbm" if bound == "hbm" else "alu", "pipe": bound, "kernel": cls, "achieved": ach,
                "peak": peak, "unit": unit, "frac": ach / peak, "traffic": traffic, "peak_source": src,
                "launches_in_profiled_pass": cn, "avg_launch_us": cms * 1e3 / max(cn, 1),
                "bytes_per_launch": cbytes / max(cn, 1), "flops_per_launch": cflops / max(cn, 1),
                "ms": cms / nprof, "hbm_frac": (cbytes / (cms / 1e3) / 1e9) / pk["hbm_gbs"]}

    active = [c for c in prof if prof[c][1] and prof[c][0] > 0]
    dom = max(active, key=lambda c: prof[c][0])
    roof = roof_of(dom)
    classes = {c: {k2: (round(v, 4) if isinstance(v, float) else v) for k2, v in roof_of(c).items()
                   if k2 in ("pipe", "ms", "launches_in_profiled_pass", "achieved", "unit", "frac", "hbm_frac")}
               for c in active}
    share = {c: round(prof[c][0] / max(sum(v[0] for v in prof.values()), 1e-9), 4) for c in prof if prof[c][1]}

    line = {
        "metric": METRIC, "value": job_tflops(flops, world, sec_step), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_step * 1e3, "seconds_per_step": sec_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if prec == "bf16" else ("f32" if prec == "fp32" else "f64"),
        "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "N": N, "leaf": m, "levels": L, "rank": r,
                   "rhs": k, "factor_precision": prec,
                   "coupling_precision": "fp64 elimination; "
                                         + ("fp64" if (args.coupling_fp64 or prec != "bf16") else "fp32")
                                         + " products of S and of the explicit inverse",
                   "residual_precision": "fp64", "solver": w["solver"], "tol": 1e-10,
                   "flops_per_step": flops, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (D, U, V = %.1f GB FP64)" % (8.0 * (m * N + 2 * r * N * L) / 1e9),
                   "kernel_classes_from": f"separate profiled pass of {nprof} steps after the timed region",
                   "restart": w.get("restart", 30 if w["solver"] == "gmres" else 0),
                   "gmres_max_iter": args.gmres_max_iter,
                   "compression_rel_err_by_level": {str(c): float(f"{e:.3g}") for c, e in
                                                    gen_stats.get("compression_rel_err", {}).items()}},
        "mixed": {"iterations": iters, "relres_reported": relres, "relres_fp64_matvec": rel_true, **err_vs_fp64,
                  "attainable_relres_bound": attainable},
        "fp64": fp64,
        "e2e": e2e,
        "adjoint": adjoint,
        "grad": grad,
        "construction": construction,
        "roofline": roof,
        "fp64_pipe_measured": fp64_meas,
        "kernel_time_share": share,
        "kernel_classes": classes,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, steps=1)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_fp64_tflops(hb, dev, stream, iters=8192, blocks_per_sm=4):
    """FP64 FMA rate of this GPU from the library's register-only probe: best
    of three launches after one warm-up, timed with CUDA events on `stream`."""
    import torch
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    best = None
    for rep in range(4):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fmas = hb.hodlr_probe_fp64_fma(iters, blocks_per_sm, out)
        b.record(stream)
        b.synchronize()
        t = a.elapsed_time(b)
        if rep and (best is None or t < best):
            best = t
    return {"tflops": 2.0 * fmas / (best / 1e3) / 1e12, "fmas": float(fmas), "ms": best,
            "blocks_per_sm": blocks_per_sm, "chains_per_thread": 8}


# ----------------------------------------------------------------- oracle (CPU) arm
def _oracle_inputs(w, log2_cap):
    """The workload's operator family at N = 2^log2_cap (same leaf, rank and
    right-hand sides), generated on the host, as the oracle's numpy arrays."""
    from synth import to_math
    ws = reduced(w, log2_cap)
    D, U, V, B = make_inputs(ws, "cpu", 0)
    return (ws["N"], ws["L"], ws["r"], ws["k"]), to_math(D, U, V, B), ws["data"]


def _oracle_step(shape, mats):
    """One pass of the oracle (factor + solve + slogdet); returns seconds."""
    from oracle.hodlr import RecursiveHODLR
    N, L, r, k = shape
    Dm, Um, Vm, Bm = mats
    t0 = time.perf_counter()
    rec = RecursiveHODLR(Dm, Um, Vm, L)
    rec.solve(Bm)
    rec.slogdet()
    return time.perf_counter() - t0


def _oracle_flops(shape):
    from oracle import costs as oc
    N, L, r, k = shape
    m = N >> L
    return oc.loop_factor_flops(N, m, r, L) + oc.loop_solve_flops(N, m, r, L, k)


def _sample_text(shape, data):
    N, L, r, k = shape
    return (f"FP64 recursive oracle (numpy/LAPACK) factor+solve+slogdet of the {data} operator at N={N}, "
            f"leaf {N >> L}, rank {r}, {k} RHS (same operator family, leaf and rank as the workload, N reduced "
            f"to bound CPU time)")


def _oracle_threads():
    """Threads the oracle's BLAS / LAPACK calls may use (numpy's thread pool
    follows the process's CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(w, steps=1):
    shape, mats, data = _oracle_inputs(w, 16)
    sec = statistics.mean(_oracle_step(shape, mats) for _ in range(steps))
    return {"value": _oracle_flops(shape) / sec / 1e12, "unit": "TFLOP/s", "cores": _oracle_threads(),
            "cpu_model": cpu_model(), "kind": "oracle", "seconds": sec, "sample": _sample_text(shape, data)}


def run_reference(args, w, rank, world):
    """The oracle as it stands on the host cores, on the same workload's
    bounded sample (N = 2^15 per step, inputs generated once), so that the
    default warm-up + timed steps end within a few minutes."""
    if rank != 0:
        return
    shape, mats, data = _oracle_inputs(w, 15)
    for _ in range(args.warmup):
        _oracle_step(shape, mats)
    sec = statistics.mean(_oracle_step(shape, mats) for _ in range(args.steps))
    val = _oracle_flops(shape) / sec / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], "cpu_sample_N": shape[0]},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": _oracle_threads(), "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": _sample_text(shape, data)},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", choices=["fp64", "fp32", "bf16"], default=None,
                    help="override the workload's factor precision")
    ap.add_argument("--solver", choices=["direct", "refine", "gmres"], default=None,
                    help="override the workload's outer solver")
    ap.add_argument("--gmres-max-iter", type=int, default=300,
                    help="FGMRES inner-iteration cap (the outer solver or the refinement's continuation)")
    ap.add_argument("--coupling-fp64", action="store_true",
                    help="BF16 factor: form the coupling products in FP64 (precision experiment)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "native":
        ap.error("--warmup must be >= 3")
    w = dict(WORKLOADS[args.workload])
    if args.prec:
        w["prec"] = args.prec
    if args.solver:
        w["solver"] = args.solver
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    try:
        run_native(args, w, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
