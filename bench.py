#!/usr/bin/env python
"""IPM benchmark: cell-steps/s of Algorithm 1 (IPM time steps) on the 1-D Euler Sod workload
(2000 cells, 3 uncertain dims, total degree 5 -> N = 56 moments x 3 variables, 6^3 = 216 Gauss nodes).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--full]

One bench step = one complete Algorithm-1 run of the workload from its initial data at t = 0 to
t_end = 0.14 (1344 time steps; each time step is the Newton solve of the dual problem in every cell,
the CFL time step and the kinetic-flux moment update, one captured CUDA graph), through ipm_run. The
headline is the mixed-precision path (Hessian on the tensor cores, everything else FP64); the plain FP64
GPU path and the FP32-factorisation mode run the same full run in the same process and are reported
beside it, with the difference of their final moments. Prints one JSON line (rank 0).
--impl reference times the CPU oracle on the host cores instead (each step a bounded sample).
With torchrun (N > 1) every rank runs an independent replica of the workload on its own GPU
(the method needs no data exchange between replicas), value = all cells updated / max time.
--full adds the long forms of the other workloads (shear layer to 200 steps, the ramp on the FP64 path
to its residual).
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
KERNELS_PER_TIME_STEP = 4    # k_order, k_newton, k_lf_combine, k_finalize (one CUDA graph per time step)
# dram__bytes_read.sum + dram__bytes_write.sum of one mixed-path k_newton launch on this workload (the
# launch of time step 691 of a whole run: 17.68 MB read, 0 written), from an ncu capture of the current
# kernel; None when no capture of the current kernel exists
NEWTON_TRAFFIC_BYTES = {"mixed": 17.68e6, "fp64": None, "mixed_f32f": None}
L2_FLUSH_BYTES = 512 << 20   # > 4x the 126 MiB L2
FP64_PROBE_N = 6144          # cuBLAS DGEMM size of the FP64 ceiling measurement
CPU_SAMPLE_STEPS = 20        # Algorithm-1 steps of the oracle in the cpu_baseline sample


def workload():
    from paper_1912_09238_gb300 import workloads
    return workloads.SOD_1D


def workload_desc(w, precision):
    return {
        "workload": (f"{w['name']}: 1-D Euler Sod tube IPM, {w['nx']} cells on [0,1], gamma 1.4, 3 uniform "
                     f"uncertain dims (rho_L, p_L, interface), total degree {w['M']} Legendre (N=56 x 3 vars), "
                     f"tensor Gauss {w['nq']}^3=216 nodes, Euler entropy (App. B), global LF kinetic flux, "
                     f"CFL {w['cfl']}, Newton tol {w['newton_tol']}; one bench step = Algorithm 1 from t=0 to "
                     f"t_end={w['t_end']} (every time step of the run)"),
        "precision": precision,
        "l2": f"flushed between timed runs ({L2_FLUSH_BYTES >> 20} MiB write on the same stream, outside the "
              "timed region); within a run the 9.7 MB state stays resident",
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


def hessian_tc_flops(N, m, Q):
    """Tensor-core flops of one mixed Hessian assembly: row tiles of 128 over the B*N rows, n_pad = N
    rounded up to 16 columns, Q rounded up to the K-chunk, three BF16 products each."""
    B = m * (m + 1) // 2
    tiles = -(-B * N // 128)
    n_pad = -(-N // 16) * 16
    kc = 32 if Q > 16 else 16
    q_pad = -(-Q // kc) * kc
    return 3 * 2.0 * tiles * 128 * n_pad * q_pad


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


def fp64_ceiling():
    """FP64 ceiling of this GPU measured here: cuBLAS DGEMM (torch.matmul on float64) of FP64_PROBE_N^3,
    best of 5 after one warm-up, CUDA events. The measured peaks file carries no FP64 figure."""
    import torch
    n = FP64_PROBE_N
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = float("inf")
    s = torch.cuda.current_stream()
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        torch.matmul(a, b)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    torch.cuda.empty_cache()
    return {"tflops": 2.0 * n ** 3 / best / 1e12,
            "source": f"measured in this run: cuBLAS DGEMM (torch.matmul, float64) {n}^3, best of 5, CUDA events"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------------------------------------
class SodRuns:
    """Complete Algorithm-1 runs of one workload in one precision on one resident context: the initial
    state is kept in pinned host buffers and restored (moments, duals, clock t = 0) before every run."""

    def __init__(self, w, precision, stream, **opt):
        import torch
        from paper_1912_09238_gb300 import ipm, workloads
        self.w = w
        self.ctx = workloads.context(w, precision=precision, **opt)
        self.ctx.set_stream(stream.cuda_stream)
        self.stream = stream
        shape = self.ctx.shape
        self.u0 = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        self.l0 = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        self.ctx.get_state(self.u0, self.l0)
        self.clock0 = ipm.ipm_clock(t=0.0, dt=0.0, steps=0, level_cap=0)
        self.cells = self.ctx.dims.n_interior

    def reset(self):
        self.ctx.set_state(self.u0, self.l0, clock=self.clock0)

    def timed_run(self, flush=None):
        """One run from t = 0 to t_end through ipm_run, CUDA-event timed on the context's stream;
        returns (seconds, time steps, last stats)."""
        import torch
        self.reset()
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(self.stream)
        s = self.ctx.run()
        b.record(self.stream)
        b.synchronize()
        if s.failed_cells or s.tc_timeouts:
            raise RuntimeError(f"dual solve failed in {s.failed_cells} cells: {s.as_dict()}")
        if s.t < self.w["t_end"] * (1 - 1e-12):
            raise RuntimeError(f"run stopped at t = {s.t}")
        return a.elapsed_time(b) / 1e3, int(s.steps), s

    def profile_run(self, with_hessian_flops):
        """One run step by step with the events inside each step's graph: per-step Newton-kernel and step
        times, Newton updates, cached checks, tensor-core Hessian phase times."""
        self.reset()
        d = self.ctx.dims
        rows = []
        while True:
            s = self.ctx.step()
            nm, _, tm = self.ctx.step_timing()
            if s.failed_cells or s.tc_timeouts:
                raise RuntimeError(f"dual solve failed: {s.as_dict()}")
            rows.append({"t": s.t, "newton_ms": nm, "step_ms": tm, "iters": s.newton_iters, "max_iters": s.max_iters,
                         "cached": s.cached_checks, "hessian_ns": s.hessian_ns, "hessian_count": s.hessian_count,
                         "flops": newton_fp64_flops(d.N, d.m, d.Q, self.cells, s.newton_iters, with_hessian_flops,
                                                    s.cached_checks)})
            if s.t >= self.w["t_end"] * (1 - 1e-12):
                return rows

    def close(self):
        self.ctx.close()


def tenths(rows):
    """Per tenth of a run's time steps: the time reached, ms per time step, Newton ms, updates and cached
    convergence checks per time step."""
    n = len(rows)
    out = []
    for k in range(10):
        sl = rows[k * n // 10:(k + 1) * n // 10]
        if not sl:
            continue
        out.append({"t": round(sl[-1]["t"], 5), "ms_per_time_step": round(statistics.mean(r["step_ms"] for r in sl), 4),
                    "newton_ms": round(statistics.mean(r["newton_ms"] for r in sl), 4),
                    "newton_updates": round(statistics.mean(r["iters"] for r in sl), 1),
                    "max_updates_per_cell": max(r["max_iters"] for r in sl),
                    "cached_checks": round(statistics.mean(r["cached"] for r in sl), 1)})
    return out


def window(rows, first, last, cells):
    sl = rows[first - 1:last]
    return {"time_steps": f"{first}..{last}", "value": cells * len(sl) / (sum(r["step_ms"] for r in sl) / 1e3),
            "unit": UNIT, "ms_per_time_step": statistics.mean(r["step_ms"] for r in sl)}


def rel_diff(a, b):
    import numpy as np
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


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
    assert torch.cuda.current_stream().cuda_stream == stream.cuda_stream != 0
    fp64 = fp64_ceiling()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    precision = args.precision
    # ---- headline: W warm-up runs, K timed runs, every run from t = 0 to t_end
    runs = SodRuns(w, precision, stream)
    for _ in range(args.warmup):
        runs.timed_run(flush)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    secs, steps_per_run, finals = [], [], []
    for _ in range(args.steps):
        sec, n, _ = runs.timed_run(flush)
        secs.append(sec)
        steps_per_run.append(n)
        finals.append(runs.ctx.get_moments())          # outside the event pair
    barrier()
    cl = clocks.stop()
    cells = runs.cells
    cell_steps = cells * sum(steps_per_run)
    value, _ = aggregate_throughput(sum(secs), cell_steps, ws, "cuda")
    head_final = finals[-1]
    runs_identical = all(np.array_equal(f, head_final) for f in finals)

    # ---- the same run step by step: per-tenth table, first-steps window, Newton-kernel roofline
    prof = runs.profile_run(precision == "fp64")
    newton_s = sum(r["newton_ms"] for r in prof) / 1e3
    flops = sum(r["flops"] for r in prof)
    achieved = flops / newton_s / 1e12
    d = runs.ctx.dims
    roofline = {"bound": "alu", "kernel": "k_newton (fused dual solve: reconstruction, closure, gradient, "
                "Hessian" + (" on tcgen05 tensor cores" if precision != "fp64" else "") +
                ", Cholesky, solves, Armijo, folded update terms)",
                "achieved": round(achieved, 4), "peak": round(fp64["tflops"], 4), "unit": "TFLOP/s",
                "frac": round(achieved / fp64["tflops"], 4), "peak_source": fp64["source"],
                "traffic": NEWTON_TRAFFIC_BYTES.get(precision),
                "measured_over": f"all {len(prof)} time steps of one full run, CUDA events around every Newton "
                                 "launch inside the step graphs",
                # moments and duals read, each cell's moment image and the duals it belongs to; the folded
                # update: two neighbours' nodal states read, two terms written
                "algorithmic_bytes_per_launch": 4 * 8 * d.n_cells * d.N * d.m
                + 8 * d.n_interior * (2 * d.m * d.Q + 2 * d.N * d.m),
                "algorithmic_fp64_flops_per_launch": round(flops / len(prof)),
                "newton_ms_mean": round(1e3 * newton_s / len(prof), 4),
                "newton_share_of_step": round(newton_s * 1e3 / sum(r["step_ms"] for r in prof), 4),
                "newton_updates_per_time_step": round(statistics.mean(r["iters"] for r in prof), 1),
                "cached_checks_per_time_step": round(statistics.mean(r["cached"] for r in prof), 1)}
    roofline_b = None
    hc = sum(r["hessian_count"] for r in prof)
    if precision != "fp64" and hc:
        hns = sum(r["hessian_ns"] for r in prof)
        per = hessian_tc_flops(d.N, d.m, d.Q)
        bf16 = measured_peaks().get("bf16_tflops_sustained")
        ach = per * hc / (hns / 1e9) / 1e12
        roofline_b = {"bound": "tensor", "kernel": "k_newton, row (b): split-BF16 Hessian on tcgen05, per SM",
                      "achieved_per_sm": round(ach, 5), "unit": "TFLOP/s",
                      "assemblies": hc, "phase_us_mean": round(hns / hc / 1e3, 3),
                      "tensor_flops_per_assembly": per}
        if bf16:
            per_sm_peak = bf16 / 152.0
            roofline_b.update({"peak_per_sm": round(per_sm_peak, 4), "frac": round(ach / per_sm_peak, 4),
                               "peak_source": "bf16_tflops_sustained of the measured peaks / 152 SMs (one CTA, "
                                              "one SM per assembly)"})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == "fp64" else "f64+bf16", "data": "synthetic",
            "config": workload_desc(w, precision), "roofline": roofline,
            "run": {"time_steps_per_run": steps_per_run[0], "ms_per_time_step": 1e3 * sum(secs) / sum(steps_per_run),
                    "p50_run_ms": 1e3 * statistics.median(secs), "max_run_ms": 1e3 * max(secs),
                    "runs_bit_identical": runs_identical,
                    "per_tenth_of_run": tenths(prof),
                    "first_time_steps": window(prof, 1, CPU_SAMPLE_STEPS, cells),
                    "steps_6_to_25": window(prof, 6, 25, cells)},
            "gpu_launches": KERNELS_PER_TIME_STEP * sum(steps_per_run), "clocks": cl}
    if roofline_b:
        line["roofline_hessian"] = roofline_b

    # ---- the other precision modes on the same full run
    if precision == "mixed" and not args.no_fp64_compare:
        comp = {}
        for name, prec, opt in (("fp64_gpu", "fp64", {}), ("mixed_f32_factor", "mixed_f32f", {}),
                                ("mixed_fma_factor", "mixed", {"factorization": 1}),
                                ("without_moment_images", "mixed", {"check_cache": 0})):
            r = SodRuns(w, prec, stream, **opt)
            r.ctx.run(20)                                   # warm-up: first time steps, then restored
            sec_c = []
            for _ in range(args.compare_runs):
                sc_, n_c, _ = r.timed_run(flush)
                sec_c.append(sc_)
            fin = r.ctx.get_moments()
            entry = {"value": cells * n_c * len(sec_c) / sum(sec_c), "unit": UNIT,
                     "ms_per_run": 1e3 * statistics.mean(sec_c), "runs": len(sec_c), "time_steps_per_run": n_c}
            if prec == "fp64":
                rows = r.profile_run(True)
                entry["per_tenth_of_run"] = tenths(rows)
                entry["first_time_steps"] = window(rows, 1, CPU_SAMPLE_STEPS, cells)
                nf = sum(x["flops"] for x in rows)
                ns_ = sum(x["newton_ms"] for x in rows) / 1e3
                entry["fp64_tflops"] = round(nf / ns_ / 1e12, 4)
                entry["frac_of_fp64_ceiling"] = round(nf / ns_ / 1e12 / fp64["tflops"], 4)
                fp64_final = fin
            comp[name] = (entry, fin)
            r.close()
        fp64_entry, fp64_final = comp["fp64_gpu"]
        fp64_entry["max_rel_diff_final_moments_mixed_vs_fp64"] = rel_diff(head_final, fp64_final)
        fp64_entry["speedup_mixed_over_fp64"] = value / fp64_entry["value"]
        line["fp64_gpu"] = fp64_entry
        e, fin = comp["mixed_f32_factor"]
        e["max_rel_diff_final_moments_vs_fp64"] = rel_diff(fin, fp64_final)
        e["speedup_over_fp64"] = e["value"] / fp64_entry["value"]
        e["what"] = ("precision mixed_f32f: tensor-core Hessian as in the headline, Cholesky factorisation and "
                     "triangular solves in FP32 (FP64 refactorisation on a non-positive FP32 pivot); gradient, "
                     "stopping test, line search and update in FP64. Not the headline: the headline keeps the "
                     "factorisation in FP64.")
        line["mixed_f32_factor"] = e
        e, fin = comp["mixed_fma_factor"]
        e["max_rel_diff_final_moments_vs_fp64"] = rel_diff(fin, fp64_final)
        e["speedup_over_fp64"] = e["value"] / fp64_entry["value"]
        e["what"] = ("the headline's mixed precision with ipm_options.factorization = 1: the Cholesky factorisation "
                     "with FP64 FMAs on the CUDA cores instead of the split factorisation (16-column FP64 panels, "
                     "trailing updates as exact digit products on the tensor cores)")
        line["mixed_fma_factor"] = e
        e, fin = comp["without_moment_images"]
        e["bit_identical_final_moments"] = bool(np.array_equal(fin, head_final))
        e["what"] = ("the headline path with ipm_options.check_cache = 0: every cell evaluates its first "
                     "convergence check instead of taking it from the moment image of its unchanged duals")
        line["without_moment_images"] = e

    # ---- end to end through the C ABI: pinned host state in, full run, pinned host state out
    shape = runs.ctx.shape
    hu = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    hl = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    e2e_runs = args.e2e_runs
    barrier()
    t0 = time.perf_counter()
    e2e_steps = 0
    for _ in range(e2e_runs):
        runs.ctx.set_state(runs.u0, runs.l0, clock=runs.clock0)     # the run's inputs, pinned host -> device
        s = runs.ctx.run()
        runs.ctx.get_state(hu, hl)                                  # the run's result, device -> pinned host
        e2e_steps += int(s.steps)
    barrier()
    e2e_value, _ = aggregate_throughput(time.perf_counter() - t0, cells * e2e_steps, ws, "cuda")
    nbytes = int(np.prod(shape)) * 8
    line["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
                   "runs": e2e_runs, "final_moments_equal_headline": bool(np.array_equal(hu, head_final)),
                   "api": "ipm_set_state (initial moments and duals from pinned host buffers, clock t = 0) + "
                          "ipm_run (to t_end) + ipm_get_state (final moments and duals into pinned host buffers); "
                          "wall clock"}
    runs.close()

    if rank == 0 and not args.no_workloads:
        line["workloads"] = workloads_bench(args)
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(args)
    if rank == 0 and not args.no_workloads:
        line["frozen_hessian"] = frozen_hessian_bench(args)
        line["collocation"] = collocation_bench(args)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------------------
def _timed_steps(ctx, n, oneshot=False, stop_residual=None, chunk=None):
    """n steps (or until the steady residual falls below stop_residual), CUDA-event timed on the
    context's stream; returns (steps, seconds, last stats, residual curve)."""
    import torch
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    done, secs, s, curve = 0, 0.0, None, []
    chunk = chunk or (100 if stop_residual else n)
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
        curve.append((done, s.residual))
        if s.failed_cells:
            raise RuntimeError(f"failed cells: {s.as_dict()}")
        if stop_residual and s.residual < stop_residual:
            break
    return done, secs, s, curve


def workloads_bench(args):
    """The other workloads on both precision paths (cell-steps/s by CUDA events): 1-D Burgers to its
    t_end; the 2-D ramp by One-Shot pseudo-time steps to its 1e-8 residual; the 2-D shear layer with
    adaptive degree 2-6 and 7^3 nodes; the Sod tube under the literal 4-variable reading of its
    configuration (the 2-D Euler system on a one-row mesh)."""
    import numpy as np
    from paper_1912_09238_gb300 import workloads
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    only = getattr(args, "only", None)
    # 1-D Burgers (200 cells, N = 6, Q = 10), Algorithm 1 to t_end = 0.11
    w = workloads.BURGERS_1D
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "burgers") else ():
        ctx = workloads.context(w, precision=prec)
        ctx.set_stream(stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s = ctx.run()
        b.record(stream)
        b.synchronize()
        secs = a.elapsed_time(b) / 1e3
        r[prec] = {"value": w["nx"] * s.steps / secs, "steps": int(s.steps), "t": s.t, "seconds": secs}
        ctx.close()
    if r:
        out["burgers1d"] = {"workload": "1-D Burgers IPM, 200 cells, N = 6, Q = 10, barrier entropy, Algorithm 1 "
                                        "from t = 0 to t_end = 0.11 (ipm_run)", "unit": UNIT, **r}
    # 2-D ramp, One-Shot to residual 1e-8
    w = workloads.RAMP_2D
    cells = w["nx"] * w["ny"]
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "ramp") else ():
        ctx = workloads.context(w, precision=prec)
        ctx.set_stream(stream.cuda_stream)
        full = prec == "mixed" or args.full
        cap = args.ramp_steps if full else args.ramp_fp64_steps
        tune = ctx.tuning()
        n, secs, s, curve = _timed_steps(ctx, cap, oneshot=True, stop_residual=w["residual_tol"] if full else None)
        r[prec] = {"value": cells * n / secs, "steps": n, "residual": s.residual, "seconds": secs,
                   "reached_tolerance": bool(s.residual < w["residual_tol"]),
                   "residual_every_800_steps": [(k, float(f"{v:.3e}")) for k, v in curve[7::8]],
                   "newton_kernel": {1: "cta_per_cell", 2: "warp_per_cell"}[tune[0]],
                   "autotune_ms": {"cta_per_cell": tune[1], "warp_per_cell": tune[2]}}
        ctx.close()
    if r:
        out["ramp2d_oneshot"] = {"workload": "2-D steady Euler, 15-degree ramp, 256 x 128 cells, 2 uniform dims, "
                                 "total degree 4 (15 x 4 moments), 5 x 5 nodes, One-Shot IPM (Algorithm 2) from the "
                                 "freestream until the steady residual (Eq. residualSteady) is below 1e-8"
                                 + ("" if args.full else f"; FP64 times its first {args.ramp_fp64_steps} steps"),
                                 "unit": UNIT, **r}
    # 2-D shear layer, adaptive degree 2..6, 7^3 nodes
    w = workloads.variant(workloads.KH_2D, M=6, nq=7)
    cells = w["nx"] * w["ny"]
    r = {}
    kh_steps = 200 if args.full else args.kh_steps
    for prec in ("mixed", "fp64", "mixed_f32f") if only in (None, "kh") else ():
        ctx = workloads.context(w, precision=prec, adapt_min_degree=2, delta_lo=2e-5, delta_hi=2e-4)
        ctx.set_stream(stream.cuda_stream)
        if args.full:
            nsteps = kh_steps if prec != "mixed_f32f" else kh_steps // 4
        else:
            nsteps = kh_steps if prec == "mixed" else max(1, kh_steps // 2)
        n, secs, s, _ = _timed_steps(ctx, nsteps, chunk=10)
        lev = ctx.get_levels().reshape(w["ny"] + 2, w["nx"] + 2)[1:-1, 1:-1]
        r[prec] = {"value": cells * n / secs, "steps": n, "seconds": secs,
                   "cells_per_degree_at_end": {str(2 + k): int(v) for k, v in
                                               enumerate(np.bincount(lev.ravel(), minlength=5))}}
        ctx.close()
    if r:
        out["kh2d_adaptive"] = {"workload": "2-D shear layer, 512 x 512 periodic, 3 uniform dims, adaptive total degree "
                                "2-6 (10-84 x 4 moments), 7^3 = 343 nodes, Algorithm 3 from the initial data "
                                f"(mixed: {kh_steps} of the 200 steps; FP64: {kh_steps if args.full else max(1, kh_steps // 2)}; "
                                f"mixed_f32f: {kh_steps // 4 if args.full else max(1, kh_steps // 2)}; mixed_f32f is the "
                                "FP32-factorisation mode, a departure from the FP64 factorisation of the headline)",
                                "unit": UNIT, **r}
    # the same with a nested Clenshaw-Curtis rule per level (default levels 2, 2, 3, 3, 3: 125 or 729 nodes)
    w = workloads.variant(workloads.KH_2D, M=6, nq=7, cc_levels=())
    r = {}
    cc_steps = max(1, kh_steps // 4)
    for prec in ("mixed", "fp64") if only in (None, "kh") else ():
        ctx = workloads.context(w, precision=prec, adapt_min_degree=2, delta_lo=2e-5, delta_hi=2e-4)
        ctx.set_stream(stream.cuda_stream)
        n, secs, s, _ = _timed_steps(ctx, cc_steps, chunk=5)
        lev = ctx.get_levels().reshape(w["ny"] + 2, w["nx"] + 2)[1:-1, 1:-1]
        r[prec] = {"value": cells * n / secs, "steps": n, "seconds": secs,
                   "cells_per_degree_at_end": {str(2 + k): int(v) for k, v in
                                               enumerate(np.bincount(lev.ravel(), minlength=5))}}
        ctx.close()
    if r:
        out["kh2d_adaptive_cc"] = {"workload": "2-D shear layer as kh2d_adaptive with a nested tensor Clenshaw-Curtis "
                                   "rule per level (degrees 2-3: 5^3 = 125 nodes, 4-6: 9^3 = 729), first "
                                   f"{cc_steps} steps", "unit": UNIT, **r}
    # Sod under the literal "56 moments x 4" reading: the 4-variable 2-D Euler system on a 2000 x 1 mesh
    # (periodic in y, v_2 = 0), Algorithm 1 to t_end
    w = workloads.SOD_1D_AS_2D
    r = {}
    for prec in ("mixed", "fp64") if only in (None, "sod_m4") else ():
        ctx = workloads.context(w, precision=prec)
        ctx.set_stream(stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s = ctx.run() if prec == "mixed" or args.full else ctx.run(args.sod_m4_fp64_steps)
        b.record(stream)
        b.synchronize()
        if s.failed_cells:
            raise RuntimeError(f"failed cells: {s.as_dict()}")
        secs = a.elapsed_time(b) / 1e3
        r[prec] = {"value": w["nx"] * s.steps / secs, "steps": int(s.steps), "t": s.t, "seconds": secs}
        ctx.close()
    if r:
        out["sod1d_m4"] = {"workload": "Sod as the headline under the literal '56 moments x 4' reading: 2-D Euler "
                           "(rho, rho v1, rho v2, E) on a 2000 x 1 Cartesian mesh, outflow left/right, periodic "
                           "bottom/top, v2 = 0, total degree 5 in 3 dims (N = 56 x 4), 216 Gauss nodes, local LF "
                           "(Rusanov) faces, CFL 0.5, to t_end 0.14" +
                           ("" if args.full else f" (FP64: its first {args.sod_m4_fp64_steps} time steps)"),
                           "unit": UNIT, **r}
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
            ctx = workloads.context(workloads.variant(w, M=N - 1, nq=Q), precision="fp64")
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
            g = workloads.collocation(workloads.variant(w, M=Q - 1, nq=Q))
            st = g.run()
            u = g.get_moments()[1:-1, :, 0]        # N = Q moments: their squares sum to the nodal variance
            rows.append({"method": "SC", "Q": Q, "steps": int(st.max_node_steps), "ms": st.elapsed_ms,
                         "E_rel_l2": err(u[:, 0], E_ref), "Var_rel_l2": err(np.sum(u[:, 1:] ** 2, axis=1), V_ref)})
            g.close()
        out[f"burgers1d_{nx}"] = {"workload": f"1-D Burgers, {nx} cells, t_end 0.11; errors against the exact "
                                              "solution's cell averages (the first-order LF error included)",
                                  "runs": rows}
    w = workloads.SOD_1D
    g = workloads.collocation(w)
    st = g.run()
    steps, _, _ = g.node_info()
    out["sod1d"] = {"workload": "1-D Sod, 2000 cells, 216 Gauss nodes (6^3), to t_end 0.14", "ms": st.elapsed_ms,
                    "node_steps_min_max": [int(steps.min()), int(steps.max())],
                    "node_cell_steps_per_s": float(steps.sum()) * w["nx"] / (st.elapsed_ms / 1e3)}
    g.close()
    return out


def frozen_hessian_bench(args):
    """The Sod workload with frozen Hessians (ipm_options.hessian_reuse 2: Cholesky factors kept per
    cell across solves, reused while they converge): both precision paths, the full run (--full) or its
    first 300 time steps."""
    from paper_1912_09238_gb300 import workloads
    import torch
    limit = None if args.full else 300
    out = {"workload": "Sod (as the headline) with hessian_reuse = 2, reuse_ratio 0.5, " +
                       ("one full run to t_end" if limit is None else f"the first {limit} time steps of a run"),
           "unit": UNIT}
    stream = torch.cuda.current_stream()
    for prec in ("mixed", "fp64"):
        ctx = workloads.context(workloads.SOD_1D, precision=prec, hessian_reuse=2)
        ctx.set_stream(stream.cuda_stream)
        it = fa = n = 0
        secs = 0.0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        while True:
            a.record(stream)
            ctx.step(sync=False)
            b.record(stream)
            s = ctx.sync_stats()
            secs += a.elapsed_time(b) / 1e3
            it += s.newton_iters
            fa += s.factorizations
            n += 1
            if s.failed_cells:
                raise RuntimeError(f"failed cells: {s.as_dict()}")
            if s.t >= workloads.SOD_1D["t_end"] * (1 - 1e-12) or (limit and n >= limit):
                break
        out[prec] = {"value": workloads.SOD_1D["nx"] * n / secs, "time_steps": n, "ms_per_time_step": 1e3 * secs / n,
                     "newton_updates_per_time_step": it / n, "factorizations_per_time_step": fa / n}
        ctx.close()
    return out


# ------------------------------------------------------------------------------------------------
def _serve(reqs, arrivals, max_active):
    """Replay the arrivals against one server; returns per-request latencies, cell-steps and the makespan."""
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
    srv.drain(3600.0)
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
    Q = (degree+1)^dims): the mixed-precision server at saturation and at Poisson rates of 0.5, 0.8 and
    1.0 x its saturation rate, and a prefix of the same requests run one after another on the plain FP64
    GPU path."""
    import numpy as np
    import torch
    from paper_1912_09238_gb300 import workloads
    n = args.serving_requests
    steps = args.serving_steps
    stream = [w for _, w in workloads.serving_requests(n, seed=1234, steps=steps)]
    reqs = [(workloads.request(w, "mixed"), w) for w in stream]
    out = {"workload": (f"{n} seeded requests (seed 1234), each 1-D Burgers or 1-D Euler, cells U[200,4000], total "
                        f"degree 2-6 in 1-3 uniform dims (N 3-84), tensor Gauss (degree+1)^dims, {steps} Algorithm-1 "
                        f"steps each, mixed precision, {args.serving_slots} slots, memory cap 90% of free HBM"),
           "requests": n}
    # saturation: everything arrives at once
    lat_sat, cs, span = _serve(reqs, [0.0] * n, args.serving_slots)
    rate_sat = n / span
    out["cell_steps"] = cs
    out["saturation"] = {"value": cs / span, "unit": UNIT, "makespan_s": span, "requests_per_s": rate_sat,
                         "p50_latency_s": float(np.percentile(lat_sat, 50)),
                         "p99_latency_s": float(np.percentile(lat_sat, 99))}
    # Poisson arrivals at fractions of the saturation rate (same requests, seeded inter-arrival times)
    for frac in (0.5, 0.8, 1.0):
        rng = np.random.default_rng(1234)
        arr = np.cumsum(rng.exponential(1.0 / (frac * rate_sat), n))
        arr -= arr[0]
        lat, cs2, span2 = _serve(reqs, list(arr), args.serving_slots)
        out[f"poisson_{frac}x"] = {"value": cs2 / span2, "unit": UNIT, "makespan_s": span2, "rate_per_s": frac * rate_sat,
                                   "p50_latency_s": float(np.percentile(lat, 50)),
                                   "p99_latency_s": float(np.percentile(lat, 99))}
    # sequential FP64 GPU: one request at a time, each to completion (a prefix of the stream)
    torch.cuda.synchronize()
    t_seq, seq_lat, cs_seq = 0.0, [], 0
    for w in stream[:args.sequential_requests]:
        t0 = time.perf_counter()
        ctx = workloads.context(w, precision="fp64")
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
        cs_seq += w["nx"] * w["steps"]
    out["sequential_fp64_gpu"] = {"value": cs_seq / t_seq, "unit": UNIT, "requests": len(seq_lat), "total_s": t_seq,
                                  "p50_latency_s": float(np.percentile(seq_lat, 50)),
                                  "p99_latency_s": float(np.percentile(seq_lat, 99)),
                                  "note": "the first requests of the stream, each alone, wall time including context "
                                          "set-up, as the server's latencies include it"}
    out["speedup_served_mixed_over_sequential_fp64"] = (cs / span) / (cs_seq / t_seq)
    return out


# ------------------------------------------------------------------------------------------------
def _oracle_dual_chunk(args):
    """Worker of the host-core baseline: the oracle's dual solve (Eq. dualIterationFunction to Eq.
    tauCrit) on one contiguous range of cells."""
    w, lam, uhat = args
    from oracle import dual as od
    prob = _oracle_chunk_problem(w)
    out = od.dual_solve(prob.space, prob.ent, lam, uhat, prob.newton)
    return out[0], out[1], out[2]


_PROB_CACHE = {}


def _oracle_chunk_problem(w, warm_only=False):
    key = w["name"]
    if key not in _PROB_CACHE:
        from tests._cases import oracle_problem
        _PROB_CACHE[key] = oracle_problem(w)
    return None if warm_only else _PROB_CACHE[key]


def _oracle_warm(w):
    _oracle_chunk_problem(w, warm_only=True)


def oracle_sample(n_steps, procs, keep_state=False):
    """Time the CPU oracle on the first n_steps Algorithm-1 steps of the full 2000-cell Sod workload from
    its initial data, with the cells' dual solves split over `procs` worker processes (the solve of each
    cell is independent; the oracle's own dual_solve runs unchanged on each range) and the rest of each
    step (nodal states, time step, moment update, boundary cells: oracle.scheme1d's functions, in the order
    of its ipm_step) in this process. Returns the seconds of each step."""
    import multiprocessing as mp
    import numpy as np
    from tests._cases import oracle_problem
    from oracle import scheme1d as s1
    w = workload()
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctxm = mp.get_context("spawn")
    secs = []
    with ctxm.Pool(procs) as pool:
        pool.map(_oracle_warm, [w] * procs)                   # workers build their tables before the clock
        bounds = np.linspace(0, st.uhat.shape[0], procs + 1).astype(int)
        for _ in range(n_steps):
            t0 = time.perf_counter()
            parts = pool.map(_oracle_dual_chunk, [(w, st.lam[a:b], st.uhat[a:b]) for a, b in zip(bounds[:-1], bounds[1:])])
            lam = np.concatenate([p[0] for p in parts])
            stat = np.concatenate([p[2] for p in parts])
            assert (stat == 0).all()
            U = s1.nodal_states(prob, lam)
            dt = s1.time_step(prob, U, st.t)
            uhat = st.uhat.copy()
            uhat[1:-1] = s1.moment_update(prob, lam, dt)
            s1.apply_bc(prob, uhat)
            lam_next = lam.copy()
            s1.apply_bc(prob, lam_next)
            st = s1.State1D(uhat=uhat, lam=lam_next, t=st.t + dt, n=st.n + 1, last_dt=dt)
            secs.append(time.perf_counter() - t0)
    out = {"cells": w["nx"], "seconds": secs, "procs": procs}
    if keep_state:
        out["uhat"] = st.uhat
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_subprocess(n_steps, procs):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_steps),
                        "--oracle-procs", str(procs)], env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline():
    procs = host_cores()
    res = _oracle_subprocess(CPU_SAMPLE_STEPS, procs)
    secs = sum(res["seconds"])
    return {"value": res["cells"] * len(res["seconds"]) / secs, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"oracle (numpy FP64) Algorithm-1 steps 1..{len(res['seconds'])} of the full {res['cells']}-cell "
                      f"Sod workload from its initial data, the cells' dual solves split over {procs} processes "
                      f"(one thread each): {secs:.1f} s; the GPU's rate on the same steps is "
                      "run.first_time_steps"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    procs = host_cores()
    res = _oracle_subprocess(args.warmup + args.steps, procs)
    times = res["seconds"][args.warmup:]
    cells = res["cells"]
    value = cells * len(times) / sum(times)
    w = workload()
    sample = (f"oracle (numpy FP64) Algorithm-1 steps {args.warmup + 1}..{args.warmup + args.steps} of the full "
              f"{cells}-cell Sod workload from its initial data, each step one bench step, the cells' dual solves "
              f"split over {procs} processes (one thread each)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {**workload_desc(w, "fp64"), "l2": "not applicable (host run)",
                       "inputs": "initial data projected by the oracle in host memory",
                       "step": "one Algorithm-1 time step of the full workload from its initial data (a bounded "
                               "sample of the run the GPU arm times whole; both report cell-steps/s)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5, help="timed full runs")
    ap.add_argument("--warmup", type=int, default=3, help="untimed full runs before them")
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed_f32f"], default="mixed")
    ap.add_argument("--full", action="store_true", help="long forms of the other workloads")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip timing the other precision modes")
    ap.add_argument("--compare-runs", type=int, default=2, help="timed full runs of each other precision mode")
    ap.add_argument("--e2e-runs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other workloads")
    ap.add_argument("--ramp-steps", type=int, default=20000, help="One-Shot step cap of the ramp workload")
    ap.add_argument("--ramp-fp64-steps", type=int, default=1000)
    ap.add_argument("--kh-steps", type=int, default=20, help="steps of the adaptive shear layer (mixed)")
    ap.add_argument("--sod-m4-fp64-steps", type=int, default=200)
    ap.add_argument("--only", choices=["burgers", "ramp", "kh", "sod_m4", "collocation", "serving"], default=None,
                    help="run only this workload's timing (no headline; for profiling)")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--serving-steps", type=int, default=10)
    ap.add_argument("--serving-slots", type=int, default=32)
    ap.add_argument("--sequential-requests", type=int, default=300)
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-procs", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample, args.oracle_procs)), flush=True)
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
        if args.only == "collocation":
            res = collocation_bench(args)
        elif args.only == "serving":
            res = serving_bench(args)
        else:
            res = workloads_bench(args)
        print(json.dumps(res), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
