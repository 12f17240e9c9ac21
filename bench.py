#!/usr/bin/env python
"""IPM benchmark: cell-steps/s of Algorithm 1 (IPM time step) on the 1-D Euler Sod workload
(2000 cells, 3 uncertain dims, total degree 5 -> N = 56 moments x 3 variables, 6^3 = 216 Gauss nodes).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

One step = one call of ipm_step: the Newton solve of the dual problem in every cell, the CFL time
step, the kinetic-flux moment update (one captured CUDA graph). The headline is the mixed-precision
path (Hessian on the tensor cores, everything else FP64); the plain FP64 GPU path is timed on the
same workload in the same run and reported beside it (--precision fp64 makes FP64 the headline),
and so is the FP32-factorisation mode (key "mixed_f32_factor").
Prints one JSON line (rank 0).
--impl reference times the CPU oracle on the host cores instead (each step a bounded sample).
With torchrun (N > 1) every rank runs an independent replica of the workload on its own GPU
(the method needs no data exchange between replicas), value = all cells updated / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IPM cell-steps/s (mixed+batched vs FP64 GPU at equal error); p50/p99 latency"
UNIT = "cell-steps/s"
FP64_PEAK_TFLOPS = 1.25      # nominal dense FP64 of a GB300 (probe: 1.19 measured with FMA chains)
KERNELS_PER_STEP = 4         # k_order, k_newton, k_lf_combine, k_finalize (one CUDA graph per step)
# dram__bytes_read.sum + dram__bytes_write.sum of one mixed-path k_newton launch on this workload,
# from an ncu capture of the current kernel (a warm step); None for the FP64 kernel (no capture yet)
NEWTON_TRAFFIC_BYTES = {"mixed": 21.58e6, "fp64": None, "mixed_f32f": None}
L2_FLUSH_BYTES = 512 << 20   # > 4x the 126 MiB L2
WINDOW = dict(nx=200, x_lo=0.45, x_hi=0.55)   # same dx as the 2000-cell mesh, around the interface


def workload():
    from paper_1912_09238_gb300 import workloads
    return workloads.SOD_1D


def workload_desc(w, precision):
    return {
        "workload": (f"{w['name']}: 1-D Euler Sod tube IPM, {w['nx']} cells on [0,1], gamma 1.4, 3 uniform "
                     f"uncertain dims (rho_L, p_L, interface), total degree {w['M']} Legendre (N=56 x 3 vars), "
                     f"tensor Gauss {w['nq']}^3=216 nodes, Euler entropy (App. B), global LF kinetic flux, "
                     f"CFL {w['cfl']}, Newton tol {w['newton_tol']}; Algorithm 1 time steps from t=0"),
        "precision": precision,
        "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write on the same stream, excluded from step times)",
        "inputs": "initial data projected on the device; state resident in HBM",
    }


# ------------------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.strip().split(",") for r in open(self.f.name).read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def newton_fp64_flops(N, m, Q, cells, iters, with_hessian, cached=0):
    """Algorithmic FP64 flops of one Newton launch: every cell evaluates the gradient (reconstruction +
    projection, 4QNm) once more than it updates, except the `cached` cells whose first check came from
    their moment image (S - u_hat and its norm, 3Nm); every update adds the Cholesky factorisation
    ((Nm)^3/3), two triangular solves (2 (Nm)^2) and the direction at the nodes (2QNm), and on the FP64
    path the Hessian (B Q N(N+1): unique entries of B blocks, Q-term dot products). Closures and
    line-search trials are not counted."""
    B = m * (m + 1) // 2
    NM = N * m
    grad_eval = 4.0 * Q * N * m
    per_update = NM ** 3 / 3.0 + 2.0 * NM ** 2 + 2.0 * Q * N * m
    if with_hessian:
        per_update += B * Q * N * (N + 1)
    return (cells - cached + iters) * grad_eval + cached * 3.0 * N * m + iters * per_update


def hessian_tc_flops(N, m, Q, iters):
    """Tensor-core flops of the mixed Hessian per launch: per update, row tiles of 128 over the B*N rows,
    n_pad = N rounded up to 16 columns, Q rounded up to the K-chunk, three BF16 products each."""
    B = m * (m + 1) // 2
    tiles = -(-B * N // 128)
    n_pad = -(-N // 16) * 16
    kc = 32 if Q > 16 else 16
    q_pad = -(-Q // kc) * kc
    return iters * 3 * 2.0 * tiles * 128 * n_pad * q_pad


def aggregate_throughput(local_seconds, units_per_rank, ws, device):
    """Whole-job throughput of weakly scaled replicas: every rank processed units_per_rank in
    local_seconds; the job took the slowest rank's time. Returns (units/s over all ranks, max seconds)."""
    secs = float(local_seconds)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([secs], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    return ws * units_per_rank / secs, secs


# ------------------------------------------------------------------------------------------------
def measure(args, precision, flush, stream, barrier, ws, **opt):
    """W warm-up + K timed Algorithm-1 steps of one precision; returns (summary dict, context)."""
    import numpy as np
    import torch
    from tests._cases import gpu_context

    w = workload()
    ctx = gpu_context(w, precision=precision, **opt)
    ctx.set_stream(stream.cuda_stream)
    d = ctx.dims
    for _ in range(args.warmup):
        flush.zero_()
        ctx.step(sync=False)
    barrier()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    newton_ms, iters, cached = [], [], []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.step(sync=False)
        ev[k][1].record(stream)
        nm, _, _ = ctx.step_timing()               # waits for this step; outside the event pair
        s = ctx.sync_stats()
        newton_ms.append(nm)
        iters.append(s.newton_iters)
        cached.append(s.cached_checks)
        if s.failed_cells or s.tc_timeouts:
            raise RuntimeError(f"dual solve failed in {s.failed_cells} cells: {s.as_dict()}")
    barrier()
    cl = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    cells = d.n_interior
    value, _ = aggregate_throughput(sum(step_ms) / 1e3, cells * args.steps, ws, "cuda")
    flops = [newton_fp64_flops(d.N, d.m, d.Q, cells, it, precision == "fp64", ch) for it, ch in zip(iters, cached)]
    newton_s = statistics.mean(newton_ms) / 1e3
    out = {"value": value, "ms_per_step": statistics.mean(step_ms),
           "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
           "newton_ms_mean": statistics.mean(newton_ms), "newton_share_of_step": sum(newton_ms) / sum(step_ms),
           "fp64_flops_per_launch": sum(flops) / len(flops),
           "fp64_tflops": (sum(flops) / len(flops)) / newton_s / 1e12,
           "newton_iters_per_step": statistics.mean(iters), "cached_checks_per_step": statistics.mean(cached),
           "clocks": cl, "cells": cells, "dims": d}
    if precision != "fp64":
        tcf = statistics.mean(hessian_tc_flops(d.N, d.m, d.Q, it) for it in iters)
        out["tensor_flops_per_launch"] = tcf
    return out, ctx


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()

    w = workload()
    stream = torch.cuda.Stream()                    # a real (non-default) stream shared by torch and libipm
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    assert torch.cuda.current_stream().cuda_stream == stream.cuda_stream != 0

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    precision = args.precision
    main, ctx = measure(args, precision, flush, stream, barrier, ws)
    d = main["dims"]
    cells = main["cells"]
    # the plain FP64 GPU path on the same workload and steps (the comparison the metric names)
    ref = None
    if precision == "mixed" and not args.no_fp64_compare:
        ref, rctx = measure(args, "fp64", flush, stream, barrier, ws)
        # equal error: both paths ran the same steps from the same initial data
        a, b = ctx.get_moments(), rctx.get_moments()
        ref["max_rel_diff_moments_vs_mixed"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        # the FP32-factorisation mode on the same steps, against the FP64 path's moments
        f32, fctx = measure(args, "mixed_f32f", flush, stream, barrier, ws)
        c = fctx.get_moments()
        f32["max_rel_diff_moments_vs_fp64"] = float(np.max(np.abs(c - b)) / np.max(np.abs(b)))
        f32["fp32_fallbacks"] = fctx.sync_stats().fp32_fallbacks
        fctx.close()
        # the headline path evaluating every convergence check (no moment images): same steps, and
        # the moments must come out bit for bit the same
        plain, pctx = measure(args, precision, flush, stream, barrier, ws, check_cache=0)
        plain["bit_identical_moments"] = bool(np.array_equal(pctx.get_moments(), a))
        pctx.close()
        rctx.close()

    roofline = {"bound": "alu", "kernel": "k_newton (fused dual solve: reconstruction, closure, gradient, "
                "Hessian" + (" on tcgen05 tensor cores" if precision == "mixed" else "") +
                ", Cholesky, solves, Armijo)", "achieved": round(main["fp64_tflops"], 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": round(main["fp64_tflops"] / FP64_PEAK_TFLOPS, 4),
                "peak_source": "nominal GB300 dense FP64 (fallback table; no FP64 figure in the measured peaks); "
                               "an FMA-chain probe measured 1.19 TFLOP/s",
                "traffic": NEWTON_TRAFFIC_BYTES[precision],
                # moments and duals read, each cell's moment image and the duals it belongs to; on 1-D
                # meshes also the folded update: two neighbours' nodal states read, two terms written
                "algorithmic_bytes_per_launch": 4 * 8 * d.n_cells * d.N * d.m
                + 8 * d.n_interior * (2 * d.m * d.Q + 2 * d.N * d.m),
                "newton_ms_mean": round(main["newton_ms_mean"], 4),
                "newton_share_of_step": round(main["newton_share_of_step"], 4),
                "algorithmic_fp64_flops_per_launch": round(main["fp64_flops_per_launch"]),
                "newton_iters_per_step": round(main["newton_iters_per_step"], 1),
                "cached_checks_per_step": round(main["cached_checks_per_step"], 1)}
    if precision == "mixed":
        roofline["tensor_bf16_flops_per_launch"] = round(main["tensor_flops_per_launch"])

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    shape = ctx.shape
    hu = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    hl = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    hu[...] = ctx.get_moments()
    hl[...] = ctx.get_duals()
    e2e_steps = args.steps
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(hu, hl)
        ctx.step(sync=False)
        ctx.get_state(hu, hl)                   # straight into the pinned buffers
    barrier()
    e2e_value, _ = aggregate_throughput(time.perf_counter() - t0, cells * e2e_steps, ws, "cuda")
    nbytes = int(np.prod(shape)) * 8
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes,
           "d2h_bytes_per_step": 2 * nbytes, "api": "ipm_set_state + ipm_step + ipm_get_state (moments and "
           "duals, pinned host buffers)"}

    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "p50_step_ms": main["p50_step_ms"], "p99_step_ms": main["p99_step_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f64+bf16", "data": "synthetic",
            "config": workload_desc(w, precision), "roofline": roofline, "e2e": e2e,
            "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": main["clocks"]}
    if ref is not None:
        line["without_moment_images"] = {
            "value": plain["value"], "unit": UNIT, "ms_per_step": plain["ms_per_step"],
            "newton_ms_mean": plain["newton_ms_mean"], "bit_identical_moments": plain["bit_identical_moments"],
            "what": "the headline path with ipm_options.check_cache = 0: every cell evaluates its first "
                    "convergence check instead of taking it from the moment image of its unchanged duals"}
        line["fp64_gpu"] = {"value": ref["value"], "unit": UNIT, "ms_per_step": ref["ms_per_step"],
                            "newton_ms_mean": ref["newton_ms_mean"],
                            "newton_iters_per_step": ref["newton_iters_per_step"],
                            "fp64_tflops": round(ref["fp64_tflops"], 4),
                            "max_rel_diff_moments_vs_mixed": ref["max_rel_diff_moments_vs_mixed"],
                            "speedup_mixed_over_fp64": main["value"] / ref["value"]}
        line["mixed_f32_factor"] = {
            "value": f32["value"], "unit": UNIT, "ms_per_step": f32["ms_per_step"],
            "p50_step_ms": f32["p50_step_ms"], "p99_step_ms": f32["p99_step_ms"],
            "newton_ms_mean": f32["newton_ms_mean"], "newton_iters_per_step": f32["newton_iters_per_step"],
            "max_rel_diff_moments_vs_fp64": f32["max_rel_diff_moments_vs_fp64"],
            "fp32_fallbacks": f32["fp32_fallbacks"], "speedup_over_fp64": f32["value"] / ref["value"],
            "what": "precision mixed_f32f: tensor-core Hessian as in the headline, Cholesky factorisation and "
                    "triangular solves in FP32 (FP64 refactorisation on a non-positive FP32 pivot); gradient, "
                    "stopping test, line search and update in FP64. Not the headline: the headline keeps the "
                    "factorisation in FP64."}
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(args)
    if rank == 0 and not args.no_workloads:
        line["workloads"] = workloads_bench(args)
    if rank == 0 and not args.no_workloads:
        line["frozen_hessian"] = frozen_hessian_bench(args)
    if rank == 0 and not args.no_workloads:
        line["collocation"] = collocation_bench(args)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------------------
def _timed_steps(ctx, n, oneshot=False, stop_residual=None):
    """n steps (or until the steady residual falls below stop_residual), CUDA-event timed on the
    context's stream; returns (steps, seconds, last stats)."""
    import torch
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    done, secs, s = 0, 0.0, None
    chunk = 50 if stop_residual else n
    while done < n:
        k = min(chunk, n - done)
        a.record(stream)
        for _ in range(k):
            (ctx.oneshot_step if oneshot else ctx.step)(sync=False)
        b.record(stream)
        b.synchronize()
        secs += a.elapsed_time(b) / 1e3
        done += k
        s = ctx.sync_stats()
        if s.failed_cells:
            raise RuntimeError(f"failed cells: {s.as_dict()}")
        if stop_residual and s.residual < stop_residual:
            break
    return done, secs, s


def workloads_bench(args):
    """The other workloads, each as a bounded run on both precision paths (cell-steps/s by CUDA events):
    1-D Burgers to its t_end; the 2-D ramp by One-Shot pseudo-time steps towards its 1e-8 residual (step
    cap); the 2-D shear layer with adaptive degree 2-6 and 7^3 nodes (a bounded number of steps)."""
    import numpy as np
    from paper_1912_09238_gb300 import workloads
    from tests._cases import gpu_context
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    only = getattr(args, "only", None)
    # 1-D Burgers (200 cells, N = 6, Q = 10), Algorithm 1 to t_end = 0.11
    w = workloads.BURGERS_1D
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "burgers") else ():
        ctx = gpu_context(w, precision=prec)
        ctx.set_stream(stream.cuda_stream)
        n, secs, s = _timed_steps(ctx, 176)
        r[prec] = {"value": w["nx"] * n / secs, "steps": n, "t": s.t, "seconds": secs}
        ctx.close()
    if r:
        out["burgers1d"] = {"workload": "1-D Burgers IPM, 200 cells, N = 6, Q = 10, barrier entropy, to t_end = 0.11",
                            "unit": UNIT, **r}
    # 2-D ramp, One-Shot towards residual 1e-8
    w = workloads.RAMP_2D
    cells = w["nx"] * w["ny"]
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "ramp") else ():
        ctx = gpu_context(w, precision=prec)
        ctx.set_stream(stream.cuda_stream)
        cap = args.ramp_steps if prec == "mixed" else min(args.ramp_steps, 200)
        tune = ctx.tuning()
        n, secs, s = _timed_steps(ctx, cap, oneshot=True, stop_residual=w["residual_tol"] if prec == "mixed" else None)
        r[prec] = {"value": cells * n / secs, "steps": n, "residual": s.residual, "seconds": secs,
                   "newton_kernel": {1: "cta_per_cell", 2: "warp_per_cell"}[tune[0]],
                   "autotune_ms": {"cta_per_cell": tune[1], "warp_per_cell": tune[2]}}
        ctx.close()
    if r:
        out["ramp2d_oneshot"] = {"workload": "2-D steady Euler, 15-degree ramp, 256 x 128 cells, 2 uniform dims, "
                                 "total degree 4 (15 x 4 moments), 5 x 5 nodes, One-Shot IPM (Algorithm 2); mixed "
                                 "runs towards residual 1e-8 (capped), FP64 times the first 200 steps",
                                 "unit": UNIT, **r}
    # 2-D shear layer, adaptive degree 2..6, 7^3 nodes
    w = workloads.variant(workloads.KH_2D, M=6, nq=7)
    cells = w["nx"] * w["ny"]
    r = {}
    for prec in ("mixed", "fp64", "mixed_f32f") if only in (None, "kh") else ():
        ctx = gpu_context(w, precision=prec, adapt_min_degree=2, delta_lo=2e-5, delta_hi=2e-4)
        ctx.set_stream(stream.cuda_stream)
        n, secs, s = _timed_steps(ctx, args.kh_steps)
        lev = ctx.get_levels().reshape(w["ny"] + 2, w["nx"] + 2)[1:-1, 1:-1]
        r[prec] = {"value": cells * n / secs, "steps": n, "seconds": secs,
                   "cells_per_degree": {str(2 + k): int(v) for k, v in enumerate(np.bincount(lev.ravel(), minlength=5))}}
        ctx.close()
    if r:
        out["kh2d_adaptive"] = {"workload": f"2-D shear layer, 512 x 512 periodic, 3 uniform dims, adaptive total degree "
                                f"2-6 (10-84 x 4 moments), 7^3 = 343 nodes, first {args.kh_steps} of the 200 steps "
                                "(mixed_f32f: the FP32-factorisation mode, a departure from the FP64 factorisation of the headline)",
                                "unit": UNIT, **r}
    # the same with a nested Clenshaw-Curtis rule per level (default levels 2, 2, 3, 3, 3: 125 or 729 nodes)
    w = workloads.variant(workloads.KH_2D, M=6, nq=7, cc_levels=())
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "kh") else ():
        ctx = gpu_context(w, precision=prec, adapt_min_degree=2, delta_lo=2e-5, delta_hi=2e-4)
        ctx.set_stream(stream.cuda_stream)
        n, secs, s = _timed_steps(ctx, max(1, args.kh_steps // 2))
        lev = ctx.get_levels().reshape(w["ny"] + 2, w["nx"] + 2)[1:-1, 1:-1]
        r[prec] = {"value": cells * n / secs, "steps": n, "seconds": secs,
                   "cells_per_degree": {str(2 + k): int(v) for k, v in enumerate(np.bincount(lev.ravel(), minlength=5))}}
        ctx.close()
    if r:
        out["kh2d_adaptive_cc"] = {"workload": "2-D shear layer as kh2d_adaptive with a nested tensor Clenshaw-Curtis "
                                   "rule per level (degrees 2-3: 5^3 = 125 nodes, 4-6: 9^3 = 729), first "
                                   f"{max(1, args.kh_steps // 2)} steps", "unit": UNIT, **r}
    return out


def burgers_exact_mean_var(nx, x_lo, x_hi, t, samples=4001, sub=32):
    """E and Var over xi ~ U[-1, 1] of the cell averages of the exact Burgers solution of the 1-D Burgers
    workload: u = 12 left of the shock x_s(xi) = 0.5 + 0.2 xi + 6.5 t (Rankine-Hugoniot speed
    (12 + 1)/2), 1 right of it; midpoint rules in xi and inside each cell."""
    import numpy as np
    dx = (x_hi - x_lo) / nx
    xi = -1.0 + (np.arange(samples) + 0.5) * 2.0 / samples
    xs = 0.5 + 0.2 * xi + 6.5 * t
    x = x_lo + (np.arange(nx)[:, None] + (np.arange(sub)[None, :] + 0.5) / sub) * dx       # (nx, sub)
    frac = np.mean(x[:, :, None] < xs[None, None, :], axis=1)                              # (nx, samples)
    u = 1.0 + 11.0 * frac
    return u.mean(axis=1), u.var(axis=1)


def collocation_bench(args):
    """Stochastic Collocation (ipm_sc_*) next to IPM on the GPU (the paper's IPM-versus-SC comparison).
    Burgers to t_end = 0.11 on 200 and 1600 cells: IPM (FP64) with (N, Q) = (3, 5), (6, 10), (10, 20)
    against SC with Q = 5, 10, 20, 40 Gauss nodes; relative L2 errors of E[u] and Var[u] against the exact
    Rankine-Hugoniot solution's cell averages, and the device time of each full run. Sod (2000 cells, 216
    nodes): the SC run to t_end = 0.14 (its time and node-cell-steps/s); the IPM Sod numbers are the
    headline's."""
    import numpy as np
    from paper_1912_09238_gb300 import workloads
    from tests._cases import gpu_collocation, gpu_context
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for nx in (200, 1600):
        w = workloads.variant(workloads.BURGERS_1D, nx=nx)
        E_ref, V_ref = burgers_exact_mean_var(nx, w["x_lo"], w["x_hi"], w["t_end"])
        dx = (w["x_hi"] - w["x_lo"]) / nx
        err = lambda a, b: float(np.sqrt(np.sum(dx * (a - b) ** 2) / np.sum(dx * b ** 2)))
        rows = []
        for N, Q in ((3, 5), (6, 10), (10, 20)):
            ctx = gpu_context(workloads.variant(w, M=N - 1, nq=Q), precision="fp64")
            ctx.set_stream(stream.cuda_stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s = ctx.run()
            ev1.record(stream)
            torch.cuda.synchronize()
            u = ctx.get_moments()[1:-1, :, 0]
            rows.append({"method": "IPM (FP64)", "N": N, "Q": Q, "steps": int(s.steps), "ms": ev0.elapsed_time(ev1),
                         "E_rel_l2": err(u[:, 0], E_ref), "Var_rel_l2": err(np.sum(u[:, 1:] ** 2, axis=1), V_ref)})
            ctx.close()
        for Q in (5, 10, 20, 40):
            g = gpu_collocation(workloads.variant(w, M=Q - 1, nq=Q))
            st = g.run()
            u = g.get_moments()[1:-1, :, 0]        # N = Q moments: their squares sum to the nodal variance
            rows.append({"method": "SC", "Q": Q, "steps": int(st.max_node_steps), "ms": st.elapsed_ms,
                         "E_rel_l2": err(u[:, 0], E_ref), "Var_rel_l2": err(np.sum(u[:, 1:] ** 2, axis=1), V_ref)})
            g.close()
        out[f"burgers1d_{nx}"] = {"workload": f"1-D Burgers, {nx} cells, t_end 0.11; errors against the exact "
                                              "solution's cell averages (the first-order LF error included)",
                                  "runs": rows}
    w = workloads.SOD_1D
    g = gpu_collocation(w)
    st = g.run()
    steps, _, _ = g.node_info()
    out["sod1d"] = {"workload": "1-D Sod, 2000 cells, 216 Gauss nodes (6^3), to t_end 0.14", "ms": st.elapsed_ms,
                    "node_steps_min_max": [int(steps.min()), int(steps.max())],
                    "node_cell_steps_per_s": float(steps.sum()) * w["nx"] / (st.elapsed_ms / 1e3)}
    g.close()
    return out


def frozen_hessian_bench(args):
    """The Sod workload with frozen Hessians (ipm_options.hessian_reuse 2: Cholesky factors kept per
    cell across solves, reused while they converge): both precision paths, 5 warm-up + 30 timed steps."""
    from paper_1912_09238_gb300 import workloads
    from tests._cases import gpu_context
    import torch
    out = {"workload": "Sod (as the headline) with hessian_reuse = 2, reuse_ratio 0.5", "unit": UNIT}
    stream = torch.cuda.current_stream()
    for prec in ("mixed", "fp64"):
        ctx = gpu_context(workloads.SOD_1D, precision=prec, hessian_reuse=2)
        ctx.set_stream(stream.cuda_stream)
        for _ in range(5):
            ctx.step(sync=False)
        it = fa = 0
        n, secs, _ = 30, 0.0, None
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(n):
            a.record(stream)
            ctx.step(sync=False)
            b.record(stream)
            s = ctx.sync_stats()
            secs += a.elapsed_time(b) / 1e3
            it += s.newton_iters
            fa += s.factorizations
        out[prec] = {"value": workloads.SOD_1D["nx"] * n / secs, "ms_per_step": 1e3 * secs / n,
                     "newton_updates_per_step": it / n, "factorizations_per_step": fa / n}
        ctx.close()
    return out


# ------------------------------------------------------------------------------------------------
def _request(w, precision):
    from paper_1912_09238_gb300 import ipm
    pr = ipm.make_problem(w["kind"], w["nx"], w["x_lo"], w["x_hi"], bc=w["bc"], cfl=w["cfl"], t_end=w["t_end"],
                          gamma=w["gamma"], x0=w["x0"], dx0=w["dx0"], left=w["left"], dleft=w.get("dleft"),
                          right=w["right"], dright=w.get("dright"))
    o = ipm.default_options(precision, newton_tol=w.get("newton_tol", 1e-10))
    return ipm.make_request(pr, w["p"], w["M"], w["nq"], w["entropy"], w.get("u_minus", 0.0), w.get("u_plus", 0.0),
                            o, max_steps=w["steps"])


def _serve(reqs, arrivals, max_active):
    """Replay the arrivals against one server; returns per-request (latency_s, cell_steps) and the makespan."""
    import numpy as np
    from paper_1912_09238_gb300 import ipm
    srv = ipm.Server(mem_cap_bytes=0, max_active=max_active)
    t0 = time.perf_counter()
    tickets = []
    for (req, w), at in zip(reqs, arrivals):
        dt = at - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(req))
    srv.drain(1800.0)
    res = [srv.poll(t, fetch=False)[0] for t in tickets]
    srv.close()
    if any(r.status != 0 for r in res):
        raise RuntimeError("served request failed: " + str([(r.status, r.error) for r in res if r.status != 0][:5]))
    lat = np.array([r.finish_s - r.submit_s for r in res])
    first = min(r.submit_s for r in res)
    last = max(r.finish_s for r in res)
    cell_steps = sum(w["nx"] * w["steps"] for _, w in reqs)
    return lat, cell_steps, last - first


def serving_bench(args):
    """Serving workload (seeded Poisson arrivals of 1-D Burgers / Euler requests of mixed sizes, N 3..84,
    Q = (degree+1)^dims): the mixed-precision server at saturation and at 0.8x its saturation rate, and the
    same requests run one after another on the plain FP64 GPU path."""
    import numpy as np
    import torch
    from paper_1912_09238_gb300 import workloads
    from tests._cases import gpu_context
    n, steps = args.serving_requests, args.serving_steps
    stream = [w for _, w in workloads.serving_requests(n, seed=1234, steps=steps)]
    reqs = [(_request(w, "mixed"), w) for w in stream]
    # saturation: everything arrives at once
    lat_sat, cs, span = _serve(reqs, [0.0] * n, args.serving_slots)
    rate_sat = n / span
    # Poisson arrivals at 0.8 x the saturation rate (same requests, seeded inter-arrival times)
    rng = np.random.default_rng(1234)
    arr = np.cumsum(rng.exponential(1.0 / (0.8 * rate_sat), n)) - 0.0
    arr -= arr[0]
    lat, cs2, span2 = _serve(reqs, list(arr), args.serving_slots)
    # sequential FP64 GPU: one request at a time, each to completion
    torch.cuda.synchronize()
    t_seq = 0.0
    seq_lat = []
    for w in stream:
        t0 = time.perf_counter()
        ctx = gpu_context(w, precision="fp64")
        for _ in range(w["steps"]):
            ctx.step(sync=False)
        s = ctx.sync_stats()
        ctx.get_moments()
        ctx.close()
        dt = time.perf_counter() - t0
        if s.failed_cells:
            raise RuntimeError("sequential FP64 request failed")
        t_seq += dt
        seq_lat.append(dt)
    return {
        "workload": (f"{n} seeded requests (seed 1234), each 1-D Burgers or 1-D Euler, cells U[200,4000], total "
                     f"degree 2-6 in 1-3 uniform dims (N 3-84), tensor Gauss (degree+1)^dims, {steps} Algorithm-1 "
                     f"steps each, mixed precision, {args.serving_slots} slots, memory cap 90% of free HBM"),
        "cell_steps": cs,
        "saturation": {"value": cs / span, "unit": UNIT, "makespan_s": span, "requests_per_s": rate_sat,
                       "p50_latency_s": float(np.percentile(lat_sat, 50)),
                       "p99_latency_s": float(np.percentile(lat_sat, 99))},
        "poisson_0.8x": {"value": cs2 / span2, "unit": UNIT, "makespan_s": span2, "rate_per_s": 0.8 * rate_sat,
                         "p50_latency_s": float(np.percentile(lat, 50)),
                         "p99_latency_s": float(np.percentile(lat, 99))},
        "sequential_fp64_gpu": {"value": cs / t_seq, "unit": UNIT, "total_s": t_seq,
                                "p50_latency_s": float(np.percentile(seq_lat, 50)),
                                "p99_latency_s": float(np.percentile(seq_lat, 99)),
                                "note": "each request alone, wall time including context set-up, as the server's "
                                        "latencies include it"},
        "speedup_served_mixed_over_sequential_fp64": (cs / span) / (cs / t_seq),
    }


# ------------------------------------------------------------------------------------------------
def oracle_step_sample(kind, n_steps):
    """Time the CPU oracle (single thread) on a bounded sample of the Sod workload.

    kind == "first_step": Algorithm 1 step 1 of the full 2000-cell workload from its initial data.
    kind == "window": n_steps consecutive Algorithm-1 steps on the 200 cells around the interface
    (same dx), from the initial data. Returns the seconds of each step."""
    from paper_1912_09238_gb300 import workloads
    from tests._cases import oracle_problem
    from oracle import scheme1d as s1
    w = workload() if kind == "first_step" else workloads.variant(workload(), **WINDOW)
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    secs = []
    for _ in range(1 if kind == "first_step" else n_steps):
        t0 = time.perf_counter()
        st = s1.ipm_step(prob, st)
        secs.append(time.perf_counter() - t0)
        assert (st.newton_status == 0).all()
    return {"cells": w["nx"], "seconds": secs}


def _oracle_subprocess(kind, n_steps=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", kind,
                        "--steps", str(n_steps)], env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline():
    res = _oracle_subprocess("first_step")
    secs = res["seconds"][0]
    return {"value": res["cells"] / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle (numpy FP64, one thread) Algorithm-1 step 1 of the full {res['cells']}-cell Sod "
                      f"workload from its initial data: {secs:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    res = _oracle_subprocess("window", args.warmup + args.steps)
    times = res["seconds"][args.warmup:]
    cells = res["cells"]
    value = cells * len(times) / sum(times)
    w = workload()
    sample = (f"oracle (numpy FP64, one thread) Algorithm-1 steps {args.warmup + 1}..{args.warmup + args.steps} "
              f"on the {cells} cells of the Sod workload around the interface (x in [0.45,0.55], same dx), "
              f"from the initial data")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {**workload_desc(w, "fp64"), "l2": "not applicable (host run)",
                       "inputs": "initial data projected by the oracle in host memory"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed_f32f"], default="mixed")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip timing the plain FP64 GPU path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-workloads", action="store_true", help="skip the Burgers / ramp / shear-layer runs")
    ap.add_argument("--ramp-steps", type=int, default=1000, help="One-Shot step cap of the ramp workload")
    ap.add_argument("--kh-steps", type=int, default=10, help="steps of the adaptive shear-layer workload")
    ap.add_argument("--only", choices=["burgers", "ramp", "kh", "collocation"], default=None,
                    help="run only this workload's timing (no JSON bench line; for profiling)")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--serving-steps", type=int, default=10)
    ap.add_argument("--serving-slots", type=int, default=32)
    ap.add_argument("--oracle-sample", choices=["first_step", "window"], default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_step_sample(args.oracle_sample, args.steps)), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        import torch
        torch.cuda.set_device(0)
        torch.cuda.set_stream(torch.cuda.Stream())
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(collocation_bench(args) if args.only == "collocation" else workloads_bench(args)), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
