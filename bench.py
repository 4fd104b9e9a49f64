"""Benchmark of the ADMM / Toeplitz-FFT hot path on GB300.

One step = one ADMM solve (Algorithm 1, fixed number of iterations, every
sub-problem S y = rhs solved to 1e-8 relative residual) of the 1024^2 x 128
workload (beta_x = 1.7, beta_y = 1.2, d = (2.0, 0.1), e = (0.5, 0.5),
gamma = 1e-6, control box [-1, 1]) in mixed precision (FDE_MIXED_DFV): float
FFT operator and preconditioner inside iterative refinement whose residuals are
double-float products while the next correction cannot finish the sub-problem
and double products otherwise, so every accepted sub-problem residual (and the
B y feeding the ADMM step) is a double product. The same solve with all
refinement products in double (FDE_MIXED), all in double-float, in FP64
throughout, with MINRES, Algorithm 2 and the matching preconditioner is timed
beside it. Inputs are resident in HBM
and each vector (1.07 GB in double) is far larger than L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADMM solve s & Toeplitz-FFT matvec GB/s at 1024²×128; mixed vs FP64 at 1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "medium", "small", "slab", "batch"])
    ap.add_argument("--admm-iters", type=int, default=3)
    ap.add_argument("--sub-tol", type=float, default=1e-8)
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 comparison, e2e and CPU baseline")
    ap.add_argument("--kernels", action="store_true",
                    help="only time the single-launch transform passes of the workload (profiling command)")
    ap.add_argument("--tiles", default=None,
                    help="fix the FFT tiles instead of autotuning: six integers 'f32 rows,axis,dfloat rows,axis,"
                         "fp64 rows,axis' (for runs under a profiler, whose serialised launches mislead the "
                         "autotuner)")
    return ap.parse_args()


def set_or_tune_tiles(prob, spec):
    """Autotune the problem's FFT tiles, or fix them from a --tiles string; returns the tiles."""
    if spec:
        v = [int(a) for a in spec.split(",")]
        if len(v) != 6:
            raise SystemExit("--tiles wants six integers")
        prob.set_tiles(v[0], v[1])
        prob.set_tiles(v[2], v[3], dfloat=True)
        prob.set_tiles(v[4], v[5], fp64=True)
    else:
        prob.autotune()
    return {"float": prob.tiles(), "dfloat": prob.tiles(dfloat=True), "fp64": prob.tiles(fp64=True),
            "autotuned": not spec}


def workload(name):
    import fde_inputs as fi
    return {"large": fi.config_large, "medium": fi.config_medium, "small": fi.config_small,
            "slab": fi.config_large_slab}[name]()


def describe(inst, admm_iters, sub_tol):
    p = inst.params
    return {
        "workload": f"{p.nx}x{p.ny}x{p.nt} two-sided space-fractional diffusion, implicit Euler; ADMM "
                    f"{admm_iters} iterations per solve, sub-solves to {sub_tol:g} relative residual",
        "nx": p.nx, "ny": p.ny, "nt": p.nt, "N": p.N, "beta": [p.beta_x, p.beta_y], "coef": [p.dp, p.dm, p.ep, p.em],
        "gamma": p.gamma, "box": {"ya": inst.ya, "yb": inst.yb, "ua": inst.ua, "ub": inst.ub},
        "delta": 1.0, "rho": 1.618,
        "precision": "mixed: float FFT operator/preconditioner PCG inside iterative refinement; refinement residuals "
                     "in double-float while the next correction cannot finish, in double for every accepted "
                     "sub-problem residual and B y (FDE_MIXED_DFV)",
        "l2": "no flush: every vector (8N bytes = %.2f GB) exceeds the 126 MB L2" % (8 * p.N / 1e9),
    }


def traffic_for(name):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None
    when the kernel sources changed since the capture (hash mismatch)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        h = hashlib.sha256()
        for fn in d["sources"]:
            with open(os.path.join(ROOT, fn), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != d["sources_sha256"]:
            return None
        return d["kernels"][name]["bytes_per_launch_full_size"]
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(inst, pcg_equiv, sample_planes=2):
    """Time the FP64 oracle's structured operators (one S application and one
    preconditioner application = one PCG iteration) on `sample_planes` time
    slices of the workload, scale to the full grid, and multiply by the number
    of PCG-iteration equivalents of one GPU solve."""
    import numpy as np
    import fde_inputs as fi
    import oracle as O
    p = inst.params
    q = fi.FdeParams(**{**p.__dict__, "nt": sample_planes})
    o = O.AdmmOptions(delta=1.0, rho=1.618)
    x = inst.ybar[:sample_planes].copy()
    O.apply_S(q, o, x[:1].copy() if sample_planes == 1 else x)  # warm caches / BLAS threads
    t0 = time.perf_counter()
    O.apply_S(q, o, x)
    O.apply_preconditioner(q, o, x)
    dt = time.perf_counter() - t0
    per_iter = dt * p.nt / sample_planes
    return {
        "value": per_iter * pcg_equiv, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
        "sample": f"one S product + one preconditioner application of the FP64 oracle on {sample_planes} of "
                  f"{p.nt} time slices ({dt:.2f} s), scaled x{p.nt / sample_planes:g} to the full grid and "
                  f"x{pcg_equiv:.1f} PCG-iteration equivalents of one solve",
        "per_pcg_iter_s": per_iter,
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst = workload(args.workload)
    # PCG-iteration equivalents of the GPU solve (measured on the GPU arm: about
    # 15 PCG iterations and 8 double matvecs per ADMM iteration at this workload)
    pcg_equiv = args.admm_iters * (15 + 4)
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(inst, pcg_equiv, sample_planes=1)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(inst, args.admm_iters, args.sub_tol), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1907_13428_gb300 as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    inst = workload(args.workload)
    p = inst.params
    prob = F.Problem(p)
    tiles = set_or_tune_tiles(prob, args.tiles)  # FFT tiles timed on this problem
    N = prob.N
    ybar = torch.as_tensor(inst.ybar.ravel(), device=dev)
    bounds = dict(ya=inst.ya, yb=inst.yb, ua=inst.ua, ub=inst.ub)
    mixed = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=args.admm_iters, fixed_iters=True, inner_tol_mode=1,
                          inner_tol=args.sub_tol, precision=F.FDE_MIXED_DFV, inner_tol_mixed=1e-4, max_pcg=500,
                          max_refine=30)
    out = {k: torch.empty(N, dtype=torch.float64, device=dev) for k in ("y", "u", "p", "zu")}
    # pinned host buffers of the end-to-end leg, allocated before the device working set grows
    hy = torch.empty(N, dtype=torch.float64).pin_memory()
    hy.copy_(torch.as_tensor(inst.ybar.ravel()))
    hout_y = torch.empty(N, dtype=torch.float64).pin_memory()
    hout_u = torch.empty(N, dtype=torch.float64).pin_memory()

    def step(opts=mixed):
        return prob.admm_solve(opts, ybar, out=out, **bounds)

    for _ in range(args.warmup):
        r = step()
    stats = r["stats"]
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = F.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        # the timed steps are the profiler's capture range (ncu --profile-from-start off)
        torch.cuda.profiler.start()
        e0.record(st)
        for _ in range(args.steps):
            r = step()
        e1.record(st)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        barrier()
    launches = F.kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ms / 1e3 / world  # seconds per solve, world solves per step (one replica per GPU)

    extras = {}
    if not args.no_extras:
        # end to end, right after the device-timed region (same clocks and power state): the
        # host-buffer entry point fde_admm_solve_host, every step copying the pinned ybar in,
        # solving and copying y and u out (copy kernels through the mapped host memory)
        hout = {"y": hout_y, "u": hout_u}
        copy_ms = []

        def e2e_step():
            rr = prob.admm_solve_host(mixed, hy, out=hout, **bounds)
            copy_ms.append((rr["stats"]["copy_in_ms"], rr["stats"]["copy_out_ms"]))
            return rr

        e2e_step()  # warm-up: first use of the staging buffer and of the host pages
        copy_ms.clear()
        n_e2e = max(2, args.steps)
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as eclk:
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            ea.record(st)
            for _ in range(n_e2e):
                rr = e2e_step()
            eb.record(st)
            torch.cuda.synchronize()
            w1 = time.perf_counter()
        te = ea.elapsed_time(eb) / 1e3 / n_e2e
        h2d_ms = sum(c[0] for c in copy_ms) / n_e2e
        d2h_ms = sum(c[1] for c in copy_ms) / n_e2e
        same = bool(torch.equal(rr["y"], r["y"].cpu()) and torch.equal(rr["u"], r["u"].cpu()))
        extras["e2e"] = {"value": te, "unit": "s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 16 * N,
                         "steps": n_e2e, "api": "fde_admm_solve_host (host buffers in and out)",
                         "wall_s": (w1 - w0) / n_e2e, "h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                         "solve_ms_in_e2e": te * 1e3 - h2d_ms - d2h_ms,
                         "result_equals_device_solve": same,
                         "host_buffers_pinned": bool(hy.is_pinned() and hout_y.is_pinned() and hout_u.is_pinned()),
                         "clocks": eclk.summary()}
        # Toeplitz-FFT matvec (float, y = B x) and the other operator units, timed alone
        def evtime(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                fn()
            b.record(st)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        x32 = ybar.float()
        y32 = torch.empty_like(x32)
        y64 = torch.empty_like(ybar)
        t_b32 = evtime(lambda: prob.matvec(x32, F.FDE_OP_B, out=y32))
        t_s32 = evtime(lambda: prob.matvec(x32, F.FDE_OP_S, mixed, out=y32))
        t_m32 = evtime(lambda: prob.precond(x32, mixed, out=y32))
        t_b64 = evtime(lambda: prob.matvec(ybar, F.FDE_OP_B, out=y64), reps=3)
        t_m64 = evtime(lambda: prob.precond(ybar, mixed, out=y64), reps=3)
        # single launches: one Kronecker factor per call (x2 pass = k_rows_reg, x1 pass = k_axis_reg)
        t_x2_64 = evtime(lambda: prob.apply_factor(ybar, 2, out=y64), reps=3)
        t_x1_64 = evtime(lambda: prob.apply_factor(ybar, 1, out=y64), reps=3)
        t_x2_32 = evtime(lambda: prob.apply_factor(x32, 2, out=y32))
        t_x1_32 = evtime(lambda: prob.apply_factor(x32, 1, out=y32))
        t_bdf = evtime(lambda: prob.matvec(ybar, F.FDE_OP_B, out=y64, dfloat=True), reps=3)
        t_x2_df = evtime(lambda: prob.apply_factor(ybar, 2, out=y64, dfloat=True), reps=3)
        t_x1_df = evtime(lambda: prob.apply_factor(ybar, 1, out=y64, dfloat=True), reps=3)
        del x32, y32, y64
        hbm, src = peaks()
        fp64_peak = F.alu_peak(F.FDE_FP64)
        fp32_peak = F.alu_peak(F.FDE_FP32)
        # Algorithmic flops per point of one pass: 4 transforms of length L per complex
        # line of two real lines at 5 L log2 L (10 log2 L per point) plus 13 for the
        # twists, symbol products and the halves' combination. Algorithmic bytes of a
        # pass: read x, write y.
        L = 1
        while L < p.ny:
            L *= 2
        flops = (10.0 * math.log2(L) + 13.0) * N
        # dominant kernel of the solve (launch-list share): the double x2 Toeplitz pass of the
        # verifying residual evaluations, bound by the double pipe (its flops at the measured
        # double FMA rate take about 40x longer than its 16N bytes at the measured copy rate)
        achieved = flops / (t_x2_64 * 1e-3) / 1e12
        gbs64 = 16.0 * N / (t_x2_64 * 1e-3) / 1e9
        extras["roofline"] = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": achieved / fp64_peak, "traffic": traffic_for("k_rows_reg_double_1024"),
                              "kernel": "k_rows_reg<double,1024>: x2 Toeplitz pass in double (one launch)",
                              "flops_per_launch": flops, "ms": t_x2_64,
                              "peak_source": "measured: fde_alu_peak_probe FMA chains, double",
                              "hbm_view": {"alg_bytes_per_launch": 16.0 * N, "gbs": gbs64, "peak": hbm,
                                           "frac": gbs64 / hbm, "peak_source": src}}
        # the float x2 pass of the PCG operator, the largest float kernel. Its arithmetic roof
        # (flops at the measured float FMA rate) lies above its memory roof (8N bytes at the
        # measured copy bandwidth), so it is reported as ALU-bound.
        ach32 = flops / (t_x2_32 * 1e-3) / 1e12
        gbs32 = 8.0 * N / (t_x2_32 * 1e-3) / 1e9
        extras["roofline_f32"] = {"bound": "alu", "achieved": ach32, "peak": fp32_peak, "unit": "TFLOP/s",
                                  "frac": ach32 / fp32_peak, "traffic": traffic_for("k_rows_reg_float_1024"),
                                  "kernel": "float x2 Toeplitz pass (k_rows_reg<float,1024>, autotuned tile; one "
                                            "launch)",
                                  "flops_per_launch": flops, "ms": t_x2_32,
                                  "peak_source": "measured: fde_alu_peak_probe FMA chains, float",
                                  "hbm_view": {"alg_bytes_per_launch": 8.0 * N, "gbs": gbs32, "peak": hbm,
                                               "frac": gbs32 / hbm, "peak_source": src}}
        alg = 8.0 * N  # read x, write y (float)
        extras["matvec"] = {"kernel": "Toeplitz-FFT matvec y = B x, float (x1 pass + x2 pass)", "ms": t_b32,
                            "alg_bytes": alg, "gbs": alg / (t_b32 * 1e-3) / 1e9, "hbm_peak": hbm,
                            "hbm_frac": alg / (t_b32 * 1e-3) / 1e9 / hbm, "hbm_peak_source": src,
                            "alu_tflops": 2 * flops / (t_b32 * 1e-3) / 1e12, "fp32_peak_tflops": fp32_peak}
        extras["operators_ms"] = {"B_f32": t_b32, "S_f32": t_s32, "precond_f32": t_m32, "B_f64": t_b64,
                                  "precond_f64": t_m64, "x2_pass_f64": t_x2_64, "x1_pass_f64": t_x1_64,
                                  "x2_pass_f32": t_x2_32, "x1_pass_f32": t_x1_32, "B_df": t_bdf,
                                  "x2_pass_df": t_x2_df, "x1_pass_df": t_x1_df}
        # all-FP64 solve with the same iteration count and sub-solve tolerance
        fp64 = F.AdmmOptions(**{**mixed.__dict__, "precision": F.FDE_FP64})
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        r64 = step(fp64)
        b.record(st)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / 1e3
        y64c, u64c = out["y"].clone(), out["u"].clone()
        r = step()
        dy = float((out["y"] - y64c).abs().max() / y64c.abs().max())
        du = float((out["u"] - u64c).abs().max() / u64c.abs().max())
        extras["fp64_compare"] = {"fp64_solve_s": t64, "mixed_solve_s": value * world, "speedup": t64 / (value * world),
                                  "mixed_vs_fp64_relerr": {"y": dy, "u": du},
                                  "fp64_stats": r64["stats"], "mixed_stats": r["stats"]}
        # the same solve with every refinement product in double (FDE_MIXED) and in double-float (FDE_MIXED_DF)
        dfo = F.AdmmOptions(**{**mixed.__dict__, "precision": F.FDE_MIXED_DF})
        step(dfo)
        torch.cuda.synchronize()
        a.record(st)
        rdf = step(dfo)
        b.record(st)
        torch.cuda.synchronize()
        tdf = a.elapsed_time(b) / 1e3
        ddy = float((out["y"] - y64c).abs().max() / y64c.abs().max())
        ddu = float((out["u"] - u64c).abs().max() / u64c.abs().max())
        dvo = F.AdmmOptions(**{**mixed.__dict__, "precision": F.FDE_MIXED})
        step(dvo)
        torch.cuda.synchronize()
        a.record(st)
        rdv = step(dvo)
        b.record(st)
        torch.cuda.synchronize()
        tdv = a.elapsed_time(b) / 1e3
        extras["refinement_products"] = {
            "headline": "FDE_MIXED_DFV (double-float steering, double-verified)",
            "all_double_FDE_MIXED_s": tdv, "headline_speedup_vs_all_double": tdv / (value * world),
            "all_double_vs_fp64_relerr": {"y": float((out["y"] - y64c).abs().max() / y64c.abs().max()),
                                          "u": float((out["u"] - u64c).abs().max() / u64c.abs().max())},
            "all_double_stats": rdv["stats"],
            "all_double_float_FDE_MIXED_DF_s": tdf, "all_double_float_vs_fp64_relerr": {"y": ddy, "u": ddu},
            "all_double_float_stats": rdf["stats"]}
        # the same solve with saddle-point sub-problems by MINRES (Section 3.3.1)
        mro = F.AdmmOptions(**{**mixed.__dict__, "inner_solver": 1, "max_pcg": 2000})
        step(mro)
        torch.cuda.synchronize()
        a.record(st)
        rmr = step(mro)
        b.record(st)
        torch.cuda.synchronize()
        tmr = a.elapsed_time(b) / 1e3
        extras["minres_compare"] = {
            "mixed_minres_solve_s": tmr, "vs_mixed_pcg": tmr / (value * world),
            "mixed_minres_vs_fp64_relerr": {"y": float((out["y"] - y64c).abs().max() / y64c.abs().max()),
                                            "u": float((out["u"] - u64c).abs().max() / u64c.abs().max())},
            "mixed_minres_stats": rmr["stats"]}
        # generalized ADMM (Algorithm 2; rho = 1, c_y = 1, c_u = 1.01 gamma) and the matching
        # Schur approximation S-hat as PCG preconditioner: the same solve otherwise
        variants = {}
        for name, kw in (("algorithm2", {"algorithm": 2, "rho": 1.0, "c_y": 1.0, "c_u": 1.01 * p.gamma}),
                         ("matching_precond", {"precond": 1})):
            vo = F.AdmmOptions(**{**mixed.__dict__, **kw})
            step(vo)
            torch.cuda.synchronize()
            a.record(st)
            rv = step(vo)
            b.record(st)
            torch.cuda.synchronize()
            variants[name] = {"solve_s": a.elapsed_time(b) / 1e3, "options": kw, "stats": rv["stats"]}
        extras["variants"] = variants
        del y64c, u64c
        if rank == 0:
            extras["cpu_baseline"] = cpu_baseline(inst, stats["pcg_iters"] + stats["fp64_matvecs"] / 2)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+double-float+f64", "data": "synthetic",
                "config": {**describe(inst, args.admm_iters, args.sub_tol), "fft_tiles_threads": tiles},
                "gpu_launches": launches,
                "clocks": clk.summary(), "solve_stats": stats}
        line.update(extras)
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """The 64 uneven instances (grids 64^2..512^2, 16..64 steps): each step solves
    every instance once (ADMM with args.admm_iters iterations, sub-solves to
    args.sub_tol) in one CUDA-graph launch per rank; with N ranks the instances
    are sharded by cost (no data-path collective) and the step time is the max
    over ranks."""
    import torch
    import torch.distributed as dist

    import fde_inputs as fi
    import paper_1907_13428_gb300 as F
    from paper_1907_13428_gb300 import sharding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    allp = fi.config_batch_params()
    parts = sharding.shard([sharding.instance_cost(p.nx, p.ny, p.nt) for p, _, _, _ in allp], world)
    mine = [allp[i] for i in parts[rank]]
    b = F.Batch([p for p, _, _, _ in mine])
    ybars = [torch.as_tensor(fi.desired_state_sine(p, sd).ravel(), device=dev) for p, _, _, sd in mine]
    ua = [a for _, a, _, _ in mine]
    ub = [c for _, _, c, _ in mine]
    opts = F.AdmmOptions(delta=1.0, rho=1.618, max_admm=args.admm_iters, inner_tol=args.sub_tol,
                         precision=F.FDE_MIXED_DFV, inner_tol_mixed=1e-4, max_refine=2, max_pcg=12)
    for _ in range(args.warmup):
        ys, us, stats = b.admm_solve(opts, ybars, ua=ua, ub=ub)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = F.kernel_launches()
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            ys, us, stats = b.admm_solve(opts, ybars, ua=ua, ub=ub)
        e1.record(st)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = sharding.max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
    launches = F.kernel_launches() - l0
    worst = max(sharding.gather_objects(max(s["max_sub_relres"] for s in stats)))
    if rank == 0:
        total_n = sum(p.N for p, _, _, _ in allp)
        line = {"metric": METRIC + " (batch workload)", "value": ms / 1e3, "unit": "s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32+double-float+f64", "data": "synthetic",
                "config": {"workload": f"{len(allp)} uneven instances (grids 64^2..512^2, 16..64 steps, "
                                       f"{total_n} points), ADMM {args.admm_iters} iterations each, sub-solves "
                                       f"to {args.sub_tol:g}, one CUDA-graph launch per rank per step",
                           "instances_per_rank": [len(x) for x in parts],
                           "l2": "no flush: the batch's vectors total %.1f GB" % (8 * total_n / 1e9)},
                "gpu_launches": launches, "graph_launches_per_step": 1, "clocks": clk.summary(),
                "max_sub_relres": worst}
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        dist.destroy_process_group()


def run_kernels(args):
    """Single launches of the transform passes on the workload (double, float and
    double-float; x2 and x1 factors): the command profiled for the roofline's traffic."""
    import torch

    import paper_1907_13428_gb300 as F
    inst = workload(args.workload)
    prob = F.Problem(inst.params)
    set_or_tune_tiles(prob, args.tiles)  # the tiles the solve uses
    x64 = torch.as_tensor(inst.ybar.ravel(), device="cuda")
    x32 = x64.float()
    y64 = torch.empty_like(x64)
    y32 = torch.empty_like(x32)
    out = {}
    for name, fn in (("x2_pass_f64", lambda: prob.apply_factor(x64, 2, out=y64)),
                     ("x1_pass_f64", lambda: prob.apply_factor(x64, 1, out=y64)),
                     ("x2_pass_f32", lambda: prob.apply_factor(x32, 2, out=y32)),
                     ("x1_pass_f32", lambda: prob.apply_factor(x32, 1, out=y32)),
                     ("x2_pass_df", lambda: prob.apply_factor(x64, 2, out=y64, dfloat=True)),
                     ("x1_pass_df", lambda: prob.apply_factor(x64, 1, out=y64, dfloat=True))):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(max(1, args.steps)):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b) / max(1, args.steps)
    tiles = {"float": prob.tiles(), "dfloat": prob.tiles(dfloat=True), "fp64": prob.tiles(fp64=True)}

    def time3(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 3

    # every tile of the two passes (threads per CTA; negative: split halves), float,
    # double-float and double
    sweep = {}
    long_rows = prob.shape[2] > 2048
    for kind, x, y, kw, rows_list, axis_list in (
            ("f32", x32, y32, {}, (256, 128), (512, 256)),
            ("df", x64, y64, {"dfloat": True}, (256, -512, -256), (256, -512)),
            ("f64", x64, y64, {"fp64": True}, (256, -512, -256), (256, -512))):
        fk = {"dfloat": True} if kind == "df" else {}
        for rows in rows_list:
            if long_rows and rows in (128, -256):
                continue
            prob.set_tiles(rows, 0, **kw)
            sweep[f"x2_{kind}_tile_{rows}"] = time3(lambda: prob.apply_factor(x, 2, out=y, **fk))
        for axis in axis_list:
            prob.set_tiles(0, axis, **kw)
            sweep[f"x1_{kind}_tile_{axis}"] = time3(lambda: prob.apply_factor(x, 1, out=y, **fk))
    prob.set_tiles(*tiles["float"])
    prob.set_tiles(*tiles["dfloat"], dfloat=True)
    prob.set_tiles(*tiles["fp64"], fp64=True)
    print(json.dumps({"kernels_ms": out, "tile_sweep_ms": sweep, "workload": describe(inst, 0, 0)["workload"],
                      "N": prob.N, "tiles": tiles}), flush=True)
    prob.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.kernels:
        run_kernels(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
