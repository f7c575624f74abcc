"""Benchmark of the IMEX finite-difference lattice Boltzmann hot path on GB300.

Workload: the 2-D four-quadrant Riemann problem, 512 x 512 cells, 8x8
Gauss-Hermite velocities for phi and for chi (128 populations per cell),
gamma = 7/5, tau = 1e-6, dt = 2.5e-5, binary64, outlet boundaries; the
quadrant states are the seeded draw ``workloads.quadrant_2d(BENCH_SEED)``.
A step is one full IMEX-SSP3(4,3,3) step: the three fused stage kernels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the problem on its own GPU (the single-grid path has no data-path
collective); value is the sum over ranks of population updates divided by
the slowest rank's time.

The reference arm (--impl reference) times the FP64 CPU oracle on all host
cores (OpenMP) on the same 512 x 512 workload; if the requested steps would
take more than about three minutes it times the first rows of the grid
instead and says so.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-velocity updates/s per IMEX step and % HBM peak; adjoint/fwd cost; mixed vs FP64"
UNIT = "cell-velocity updates/s"

# Algorithmic binary64 flops per population and launch of each fused stage
# kernel (FMA = 2): two MP-9 interface values per population (x and y), each
# 17 (9-point F^L) + 2 (differences) + 2 (F^MP) + 3 (limiter test) = 24; the
# flux difference 5; the stage's explicit part, moments and relaxation
# (stage 3: 12 + 4 + 4; stage 4: 8 + 4 + 4 and final: 4 + 4 + 4, their
# explicit parts taking the previous stage's D_i terms).  The limited MP
# branch, divisions and per-cell equilibrium factors are not counted.
FLOPS_PER_POP = {"stage3": 48 + 5 + 20, "stage4": 48 + 5 + 16, "final": 48 + 5 + 12}
# The kernels are bound by GB300's binary64 pipe, which executes one add,
# multiply or fused multiply-add per lane slot (2 slots per SM and clock), so
# the roofline counts binary64 operations, not flops.  Algorithmic operations
# per population and launch: one MP-9 interface value per axis (x and y), 15
# each (the new difference, the 8-term stencil, the curvature, the two DM
# candidates, the MD and LC bounds, the clamped result); the flux difference 4
# (two differences, a multiply, an fma); then the stage's explicit part,
# moment sums and relaxation: stage 3 6 + 4 + 3, stage 4 4 + 4 + 3, final
# 2 + 4 + 3.  The tiles' extra interface per line, the per-cell equilibrium
# factors and divisions are not counted.
FP64_OPS_PER_POP = {"stage3": 30 + 4 + 13, "stage4": 30 + 4 + 11, "final": 30 + 4 + 9}
# Algorithmic HBM bytes per population and launch (binary64): arrays read and
# written once each by the kernel (stage 3: F2, F, D -> F3, A4, Af, D3;
# stage 4: F3, A4, Af, D3 -> F4, Af, D4; final: F4, Af, D4 -> F, D, F2).
BYTES_PER_POP = {"stage3": 7 * 8, "stage4": 7 * 8, "final": 6 * 8}
# Mixed precision (binary32 arrays, 4 B per population and array; each array
# a kernel touches counted once): stage 3 reads sh, fa, D, sl and writes r3l,
# a4l, afl, D, fb; stage 4 reads sh, fb, D, a4l, afl and writes a4l, afl, D,
# fc; the final stage reads sh, fc, D, afl and writes the next state's nh, nl,
# D, fa.  (Each kernel's second, per-cell pass re-reads two arrays it has
# just read or written; those re-reads are not counted.)  Per cell: the
# binary64 moment sums of sh (4 doubles), read by stages 3 and 4 and written
# by the final stage: 32 / 128 B per population for the 8x8 lattice.
MIXED_CELL_BYTES_PER_POP = 4 * 8 / 128
BYTES_PER_POP_MIXED = {k: 4 * n + MIXED_CELL_BYTES_PER_POP
                       for k, n in (("stage3", 9), ("stage4", 9), ("final", 8))}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of the stage kernels on this workload, valid for the kernel sources
# whose SHA-256 (over STAGE_KERNEL_SOURCES in that order, comments removed) is
# recorded here; reported as null once that code differs.
TRAFFIC_SRC_SHA256 = "26a80a91309240882998c72494ffb1139e90bb407389d2e7ec2ebd6f8c04ab2c"
TRAFFIC_BYTES = {
    "fp64": {"stage3": 2373754368, "stage4": 2352021504, "final": 1849603072},
    "mixed": {"stage3": 1484165888, "stage4": 1478261760, "final": 1342670592},
}


# The sources the stage kernels are compiled from.
STAGE_KERNEL_SOURCES = ("fdlb_device.cuh", "fdlb_internal.h", "fdlb_kernels.cu", "fdlb_mixed.cu",
                        "fdlb_mp9.cuh", "fdlb_tile.cuh")


def _kernel_sources_sha256(root=None):
    """SHA-256 of the stage kernels' sources with // comments and blank lines
    removed, so that a comment edit keeps the recorded traffic."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in STAGE_KERNEL_SOURCES:
        with open(os.path.join(root or ROOT, "paper_1909_08390_gb300", "csrc", name)) as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def _traffic(kind, stage):
    if _kernel_sources_sha256() != TRAFFIC_SRC_SHA256:
        return None
    return TRAFFIC_BYTES[kind][stage]


# binary64 peak: 152 SMs x 2 DFMA lanes/clk/SM (the 1.25 TFLOP/s nominal
# figure of GB300 at 2070 MHz) x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_GOPS = 152 * 2 * 2.07e9 / 1e9  # binary64 operations per second


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 6:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[2:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist_setup():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_quadrant_problem(O, W, rows: int):
    """The benchmark workload restricted to its first `rows` rows (all 512
    rows: the whole workload), for the oracle."""
    wl = W.quadrant_2d(W.BENCH_SEED)
    y1 = rows / wl.ny
    pr = O.Problem(d=2, nx=wl.nx, ny=rows, x0=wl.x0, x1=wl.x1, y0=0.0, y1=y1, Qphi=wl.Qphi,
                   Qchi=wl.Qchi, gamma=wl.gamma, tau=wl.tau, dt=wl.dt)
    return wl, pr, O.init_states(pr, wl.states, wl.xsplit, 0.5 * y1)


def cpu_baseline_sample(steps: int = 5, rows: int = 64, threads: int = 1):
    """Oracle timing (FP64, host) on the first `rows` rows of the workload with
    `threads` OpenMP threads: updates/s, seconds, sample description."""
    from oracle import oracle as O
    from paper_1909_08390_gb300 import workloads as W
    before = O.set_threads(0)
    used = O.set_threads(threads)
    try:
        wl, pr, F0 = _oracle_quadrant_problem(O, W, rows)
        t0 = time.perf_counter()
        O.step(pr, F0, steps)
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(before)
    units = pr.npop * wl.nx * rows * steps
    return units / dt, dt, used, (f"{steps} oracle steps on {wl.nx}x{rows} cells x {pr.npop} "
                                  f"populations, {used} thread(s)")


def run_reference(args, world, rank):
    """The reference arm: the FP64 CPU oracle as it stands, on all host cores,
    on the whole 512 x 512 workload (on fewer rows, stated, if the requested
    steps would not finish within about three minutes)."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1909_08390_gb300 import workloads as W
    O.build()
    cores = _host_cores()
    O.set_threads(cores)
    rows = 512
    wl, pr, F = _oracle_quadrant_problem(O, W, rows)
    t0 = time.perf_counter()
    F = O.step(pr, F, 1)
    per_step = time.perf_counter() - t0
    if per_step * (args.steps + args.warmup) > 180.0:
        rows = max(8, int(512 * 180.0 / (per_step * (args.steps + args.warmup))) // 8 * 8)
        wl, pr, F = _oracle_quadrant_problem(O, W, rows)
    F = O.step(pr, F, args.warmup)
    t0 = time.perf_counter()
    F = O.step(pr, F, args.steps)
    el = time.perf_counter() - t0
    units = pr.npop * wl.nx * rows * args.steps
    value = units / el
    sample = (f"{args.steps} oracle steps on {wl.nx}x{rows} cells"
              f"{'' if rows == 512 else f' (first {rows} rows)'} x {pr.npop} populations, "
              f"{cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"quadrant_2d_s{W.BENCH_SEED} 512x512, 8x8 velocities (128 pops), "
                               "gamma=1.4, tau=1e-6, dt=2.5e-5, FP64" +
                               ("" if rows == 512 else f", oracle sample of {rows} rows"),
                   "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def adjoint_cost(fdlb, stream):
    """Times, on the 2048-cell differentiable run (Q = 8, gamma = 7/5,
    tau = 1e-5, dt = 2e-5, 2000 steps, checkpoints every 50): the plain
    forward steps, the checkpointed forward and the reverse pass (segment
    recomputation + the three adjoint stage kernels per step); median of 3."""
    import torch
    from paper_1909_08390_gb300 import workloads as W
    run = W.adjoint_1d()
    spec = run.spec()
    prm = torch.as_tensor(run.params(), device="cuda")
    n0, u0, T0 = fdlb.blended_fields(prm, run.nx, run.x0, run.x1, run.width)
    ctx, _ = fdlb._field_context(spec, run.gamma, run.tau, n0, u0, T0)
    try:
        P = fdlb.fdlb_npop(ctx)
        start = torch.empty((P, run.nx), dtype=torch.float64, device="cuda")
        fdlb.fdlb_get_state(ctx, start, True)
        ck = torch.empty((run.nsteps // run.every + 1, P, run.nx), dtype=torch.float64,
                         device="cuda")
        Fbar = torch.zeros((P, run.nx), dtype=torch.float64, device="cuda")
        nbar = torch.ones(run.nx, dtype=torch.float64, device="cuda")

        def timed(fn, reps=3):
            ms = []
            for _ in range(reps):
                fdlb.fdlb_set_state(ctx, start, True)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return statistics.median(ms)

        fdlb.fdlb_step(ctx, 64)  # warm-up (graph capture, first launches)
        fwd = timed(lambda: fdlb.fdlb_step(ctx, run.nsteps))
        ckf = timed(lambda: fdlb.fdlb_forward_ckpt(ctx, run.nsteps, run.every, ck))

        def reverse():
            # dLoss/dF of the loss sum(n): the library's moment adjoint
            fdlb.fdlb_moments_adjoint(ctx, nbar, None, None, None, Fbar)
            fdlb.fdlb_adjoint(ctx, run.nsteps, run.every, ck, Fbar)

        reverse()  # work space allocation
        rev = timed(reverse)
    finally:
        fdlb.fdlb_destroy(ctx)
    return {
        "workload": "1-D blended shock tube, 2048 cells, Q=8 (16 populations), gamma=7/5, "
                    "tau=1e-5, dt=2e-5, 2000 steps, checkpoints every 50, FP64",
        "forward_ms_per_step": fwd / run.nsteps,
        "checkpointed_forward_ms_per_step": ckf / run.nsteps,
        "reverse_ms_per_step": rev / run.nsteps,
        "reverse_over_forward": rev / fwd,
        "forward_plus_reverse_over_forward": (ckf + rev) / fwd,
        "gpu_launches_reverse_per_step": 6,
    }


def explicit_comparison(fdlb, stream):
    """Sec. VI's claim on the paper's shock tube (Q = (5, 3), 400 nodes,
    tau = 1e-5, t = 0.15): the IMEX step at dt/tau = 50 (300 steps) against
    the fully explicit SSP-RK3 comparator at dt/tau = 1 (15000 steps), both
    through the same fused kernels; wall time of the runs and the largest
    density difference between them."""
    import numpy as np
    import torch
    from paper_1909_08390_gb300 import workloads as W
    out = {}
    dens = {}
    for name, dt, tab in (("imex", 5e-4, None),
                          ("explicit_ssprk3", 1e-5,
                           fdlb.fdlb_named_tableau(fdlb.FDLB_TABLEAU_EXPLICIT_SSPRK3))):
        wl = W.sod_paper(S=400, dt=dt)
        with fdlb.Solver.from_workload(wl, tableau=tab, stream=stream) as s:
            ms = []
            for _ in range(3):
                s.init_riemann(wl.states, wl.xsplit)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(wl.nsteps)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            dens[name] = s.moments()[0]
        out[name] = {"dt": dt, "dt_over_tau": dt / wl.tau, "steps": wl.nsteps,
                     "ms_to_t": statistics.median(ms)}
    return {
        "workload": "Sod shock tube, 400 nodes, Q=(5,3) (8 populations), gamma=7/5, tau=1e-5, "
                    "t=0.15, FP64",
        **out,
        "speedup": out["explicit_ssprk3"]["ms_to_t"] / out["imex"]["ms_to_t"],
        "max_abs_density_difference": float(np.abs(dens["imex"] - dens["explicit_ssprk3"]).max()),
    }


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1909_08390_gb300 import build as B, fdlb, workloads as W

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    _barrier(world)
    fdlb.load()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    wl = W.quadrant_2d(W.BENCH_SEED)
    s = fdlb.Solver.from_workload(wl, stream=stream)
    s.init_riemann(wl.states, wl.xsplit, wl.ysplit)
    P, N = s.P, s.N
    units_per_step = P * N
    launches_per_step = fdlb.fdlb_launches_per_step(s.ctx)

    # warm-up
    fdlb.fdlb_step(s.ctx, args.warmup)
    torch.cuda.synchronize()

    # timed region: K steps, per-kernel CUDA events recorded inside the library
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        stage_ms = fdlb.fdlb_step_timed(s.ctx, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        _barrier(world)
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms = _max_over_ranks(world, elapsed_ms)
    value = world * units_per_step * args.steps / (elapsed_ms * 1e-3)

    # roofline of the dominant stage kernel
    names = ["stage3", "stage4", "final"]
    top = max(range(3), key=lambda i: stage_ms[i])
    per_launch_ms = stage_ms[top] / args.steps
    flops = FLOPS_PER_POP[names[top]] * units_per_step
    achieved_tflops = flops / (per_launch_ms * 1e-3) / 1e12
    ops = FP64_OPS_PER_POP[names[top]] * units_per_step
    achieved_gops = ops / (per_launch_ms * 1e-3) / 1e9
    hbm_bytes = BYTES_PER_POP[names[top]] * units_per_step
    peaks = _load_peaks()
    # the binary64 pipe's measured ceiling: independent DFMA chains on every SM
    # (fdlb_measure_fp64_pipe), taken after the timed region
    dfma_rate, _ = fdlb.fdlb_measure_fp64_pipe(stream)
    meas_gops = dfma_rate / 1e9
    roofline = {
        "bound": "alu", "kernel": f"stage_kernel<2,8,8,{names[top]}>",
        "achieved": achieved_gops, "peak": meas_gops, "unit": "G binary64 op/s",
        "frac": achieved_gops / meas_gops,
        "peak_source": "measured: fdlb_measure_fp64_pipe, 8 independent DFMA chains per thread, "
                       "2048 threads per SM (MEASURED_PEAKS.json has no binary64 figure)",
        "peak_nominal": FP64_PEAK_GOPS, "frac_of_nominal": achieved_gops / FP64_PEAK_GOPS,
        "peak_nominal_source": "152 SMs x 2 binary64 lanes/clk x 2.07 GHz",
        "traffic": _traffic("fp64", names[top]),
        "algorithmic_ops_per_launch": ops,
        "achieved_tflops": achieved_tflops, "tflops_frac": achieved_tflops / FP64_PEAK_TFLOPS,
        "algorithmic_flops_per_launch": flops,
        "avg_launch_ms": per_launch_ms,
        "stage_ms_per_step": {n: v / args.steps for n, v in zip(names, stage_ms)},
        "hbm_achieved_gbs": hbm_bytes / (per_launch_ms * 1e-3) / 1e9,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }

    # mixed precision on the same workload and step window: binary32
    # populations, binary64-accurate moments; error against the binary64 run
    mixed = None
    if not args.no_mixed:
        m = fdlb.Solver.from_workload(wl, precision=fdlb.FDLB_MIXED, stream=stream)
        m.init_riemann(wl.states, wl.xsplit, wl.ysplit)
        fdlb.fdlb_step(m.ctx, args.warmup)
        torch.cuda.synchronize()
        e0m, e1m = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(world)
        e0m.record(stream)
        mstage = fdlb.fdlb_step_timed(m.ctx, args.steps)
        e1m.record(stream)
        torch.cuda.synchronize()
        mixed_ms = _max_over_ranks(world, e0m.elapsed_time(e1m))
        mt = max(range(3), key=lambda i: mstage[i])
        m_launch_ms = mstage[mt] / args.steps
        m_bytes = BYTES_PER_POP_MIXED[names[mt]] * units_per_step
        m_gbs = m_bytes / (m_launch_ms * 1e-3) / 1e9
        # both runs are now at step warmup + steps from the same initial state
        def fields(sol):
            n, ux, uy, T = sol.moments()
            return n, ux, uy, T
        fn, fu, fv, fT = fields(s)
        mn, mu, mv, mT = fields(m)
        relerr = lambda a, b, floor=0.0: float(np.abs(a - b).max() / max(np.abs(b).max(), floor))
        mixed = {
            "value": world * units_per_step * args.steps / (mixed_ms * 1e-3), "unit": UNIT,
            "dtype": "f32 storage/advection, f64-accurate moments",
            "ms_per_step": mixed_ms / args.steps,
            "speedup_vs_fp64": elapsed_ms / mixed_ms,
            "err_vs_fp64": {"n": relerr(mn, fn), "u": relerr(mu, fu, 1.0),
                            "v": relerr(mv, fv, 1.0), "T": relerr(mT, fT),
                            "after_steps": args.warmup + args.steps},
            "roofline": {"bound": "hbm", "kernel": f"mixed_stage_kernel<2,8,8,{names[mt]}>",
                         "achieved": m_gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": (m_gbs / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "traffic": _traffic("mixed", names[mt]), "avg_launch_ms": m_launch_ms,
                         "stage_ms_per_step": {n: v / args.steps for n, v in zip(names, mstage)},
                         # every stage kernel's fraction (the line's frac is the slowest's)
                         "frac_by_stage": {
                             n: (BYTES_PER_POP_MIXED[n] * units_per_step / (v / args.steps * 1e-3)
                                 / 1e9 / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None
                             for n, v in zip(names, mstage)}},
            "gpu_launches": launches_per_step * args.steps,
        }
        # accuracy over a long run: both runs continued, untimed, to
        # --long-steps steps from the same initial state
        if args.long_steps > args.warmup + args.steps:
            more = args.long_steps - args.warmup - args.steps
            fdlb.fdlb_step(s.ctx, more)
            fdlb.fdlb_step(m.ctx, more)
            torch.cuda.synchronize()
            (fn, fu, fv, fT), (mn, mu, mv, mT) = fields(s), fields(m)
            l1err = lambda a, b, floor=0.0: float(np.abs(a - b).sum() / max(np.abs(b).sum(), floor * b.size))
            mixed["err_vs_fp64_long"] = {
                "after_steps": args.long_steps,
                "max": {"n": relerr(mn, fn), "u": relerr(mu, fu, 1.0), "v": relerr(mv, fv, 1.0),
                        "T": relerr(mT, fT)},
                "l1": {"n": l1err(mn, fn), "u": l1err(mu, fu, 1.0), "v": l1err(mv, fv, 1.0),
                       "T": l1err(mT, fT)}}
        m.close()

    # batched 1-D problems (512 two-state problems of uneven length and
    # gamma, binary32 storage, autotuned tiles, graph replay) against the
    # single-problem binary64 path run problem by problem
    batched = None
    if not args.no_batched:
        # the problems are independent: under torchrun each rank takes its own
        # share (no collective on the data path; max of the ranks' times)
        allp = W.batched_problems(0)
        total_cells = sum(q["nx"] for q in allp)
        probs = [allp[i] for i in W.shard_problems([q["nx"] for q in allp], rank, world)]
        bnx = [q["nx"] for q in probs]
        bgm = [q["gamma"] for q in probs]
        bst = np.array([q["states"] for q in probs])
        bs = fdlb.BatchSolver(bnx, bgm, tau=1e-6, dt=2e-5, precision=fdlb.FDLB_MIXED, stream=stream)
        bs.init_riemann(bst)
        variant, ctas = bs.autotune(trial_steps=2)
        bs.step(args.warmup, allow_unstable=True)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(world)
        b0.record(stream)
        bs.step(args.steps, allow_unstable=True)
        b1.record(stream)
        torch.cuda.synchronize()
        b_ms = _max_over_ranks(world, b0.elapsed_time(b1))
        b_units = bs.P * total_cells * args.steps  # all ranks' problems
        b_gbs = ((4 * 26 + 3 * 4 * 8 / 16) * bs.P * total_cells / world
                 / (b_ms / args.steps * 1e-3) / 1e9)
        flags = bs.status()
        # cells of the members that stayed valid (all ranks): the unstable
        # members' cells are stepped too, but their results are not valid
        stable_cells = _sum_over_ranks(world, float(sum(n for n, f in zip(bnx, flags) if f == 0)))
        bs.close()
        # sequential binary64 single-problem contexts on every 16th problem
        # (one GPU only: the comparison is with the batch on the same GPU)
        seq_ms, seq_cells = 0.0, 0
        for i in range(0, len(probs) if world == 1 else 0, 16):
            with fdlb.Solver(d=1, nx=bnx[i], x0=-0.5, x1=0.5, Qphi=8, Qchi=8, gamma=bgm[i],
                             tau=1e-6, dt=2e-5, stream=stream) as one:
                one.init_riemann(bst[i], 0.0)
                try:
                    one.step(args.warmup)
                except fdlb.FdlbError:
                    pass
                torch.cuda.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                try:
                    one.step(args.steps)
                except fdlb.FdlbError:
                    pass
                s1.record(stream)
                torch.cuda.synchronize()
                seq_ms += s0.elapsed_time(s1)
                seq_cells += bnx[i]
        seq_ms_all = seq_ms * (total_cells / seq_cells) if seq_cells else None
        batched = {
            "workload": "512 two-state 1-D problems, Nx ~ U[256,4096] (total %d cells), gamma ~ "
                        "U[1.1,5/3], Q=8 (16 populations), tau=1e-6, dt=2e-5" % total_cells,
            "scaling": "strong (the 512 problems dealt out over the ranks)",
            "problems_per_rank": len(probs),
            "value": bs.P * stable_cells * args.steps / (b_ms * 1e-3), "unit": UNIT,
            "value_scope": "updates of the members that stayed valid",
            "value_all_members": b_units / (b_ms * 1e-3),
            "dtype": "f32 storage/advection, f64-accurate moments",
            "ms_per_step": b_ms / args.steps,
            "sequential_fp64_ms_per_step": seq_ms_all / args.steps if seq_ms_all else None,
            "speedup_vs_sequential_fp64": seq_ms_all / b_ms if seq_ms_all else None,
            "sequential_sample": "every 16th problem (32), scaled by cell count",
            "tiling": {"cells_per_tile": [127, 63, 255][variant], "ctas_per_sm": ctas},
            "unstable_members": int(_sum_over_ranks(world, float((flags != 0).sum()))),
            # whole-step algorithmic HBM bytes of the three kernels: 26
            # population-array accesses of 4 B (each array a kernel touches,
            # once) and, per kernel and cell, the 4 binary64 moment sums of sh
            # (32 / 16 B per population)
            "roofline": {
                "bound": "hbm", "scope": "whole step (3 kernels), per GPU",
                "achieved": b_gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": b_gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "gpu_launches": 3 * args.steps,
        }

    # discrete adjoint (1-D, binary64): the differentiable 2048-cell run of
    # 2000 steps with checkpoints every 50 steps; cost of the reverse pass
    # against the plain forward steps of the same problem
    adjoint = None
    if not args.no_adjoint and world == 1:
        adjoint = adjoint_cost(fdlb, stream)

    # Sec. VI: IMEX at dt/tau = 50 against the fully explicit comparator
    comparator = None
    if not args.no_adjoint and world == 1:
        comparator = explicit_comparison(fdlb, stream)

    # end to end through the C ABI with host buffers: per step, upload the
    # state from pinned host memory, advance one step, read the moments back.
    host_state = torch.empty(s.shape, dtype=torch.float64, pin_memory=True)
    fdlb.fdlb_get_state(s.ctx, host_state.numpy(), False)
    sh = s.shape[1:]
    mom = [torch.empty(sh, dtype=torch.float64, pin_memory=True) for _ in range(4)]
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fdlb.fdlb_set_state(s.ctx, host_state.numpy(), False)
        fdlb.fdlb_step(s.ctx, 1)
        fdlb.fdlb_moments(s.ctx, mom[0].numpy(), mom[1].numpy(), mom[2].numpy(), mom[3].numpy(),
                          False)
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": world * units_per_step * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(host_state.numel() * 8),
           "d2h_bytes_per_step": int(4 * N * 8), "steps": e2e_steps}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # all host cores on the whole grid, and one core on its first 64 rows
        v, secs, used, sample = cpu_baseline_sample(steps=5, rows=512, threads=_host_cores())
        v1, secs1, _, sample1 = cpu_baseline_sample(steps=5, rows=64, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
               "seconds": secs,
               "single_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1,
                               "seconds": secs1}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded four-quadrant Riemann states)",
        "config": {"workload": f"quadrant_2d_s{W.BENCH_SEED} 512x512, 8x8 velocities (128 pops), "
                               "gamma=1.4, tau=1e-6, dt=2.5e-5, FP64",
                   "cells": int(N), "populations": int(P), "parallelism": f"replicas{world}",
                   "l2": "working set 1.6 GB > 129 MB L2 (no flush needed)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "mixed": mixed,
        "batched": batched, "adjoint": adjoint, "explicit_comparator": comparator,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_mixed_at_scale(args):
    """The mixed path (binary32 populations) on the benchmark seed's quadrant
    problem at `--scale-n`^2 cells x 128 populations (2048: about 2.1 GB per
    array) for `--scale-steps` steps, timed, with its n, u, v, T difference
    from the same run in binary64 on the GPU (max-norm and L1, relative).  A
    third run, binary64 from the initial state rounded to binary32, shows how
    far the problem itself carries a binary32-sized perturbation.  Not part of
    the default line (the binary64 run at 2048^2 takes about 0.19 s per step)."""
    import numpy as np
    import torch

    from paper_1909_08390_gb300 import build as B, fdlb, workloads as W
    B.build()
    fdlb.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.scale_n
    wl = W.quadrant_2d(W.BENCH_SEED, n=n)
    res, ms = {}, {}
    runs = (("mixed", fdlb.FDLB_MIXED, False), ("fp64", fdlb.FDLB_FP64, False),
            ("fp64_from_binary32_start", fdlb.FDLB_FP64, True))
    for name, prec, rounded in runs:
        with fdlb.Solver.from_workload(wl, precision=prec, stream=stream) as s:
            s.init_riemann(wl.states, 0.5, 0.5)
            if rounded:
                s.set_state(s.state().astype(np.float32).astype(np.float64))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(args.scale_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[name] = e0.elapsed_time(e1)
            res[name] = s.moments()

    def diff(a, b):
        out = {}
        for k, x, y, floor in zip("nuvT", a, b, (0.0, 1.0, 1.0, 0.0)):
            out[k] = {"max": float(np.abs(x - y).max() / max(np.abs(y).max(), floor)),
                      "l1": float(np.abs(x - y).sum() / max(np.abs(y).sum(), floor * y.size))}
        return out

    units = n * n * 128 * args.scale_steps
    print(json.dumps({
        "workload": "quadrant_2d_s%d %dx%d, 8x8 velocities (128 pops), gamma=1.4, tau=1e-6, "
                    "dt=2.5e-5" % (W.BENCH_SEED, n, n),
        "steps": args.scale_steps,
        "mixed": {"ms_per_step": ms["mixed"] / args.scale_steps,
                  "value": units / (ms["mixed"] * 1e-3), "unit": UNIT},
        "fp64": {"ms_per_step": ms["fp64"] / args.scale_steps,
                 "value": units / (ms["fp64"] * 1e-3), "unit": UNIT},
        "mixed_vs_fp64": diff(res["mixed"], res["fp64"]),
        "fp64_binary32_start_vs_fp64": diff(res["fp64_from_binary32_start"], res["fp64"]),
    }), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--long-steps", type=int, default=2000,
                    help="continue the binary64 and mixed runs (untimed) to this many steps and "
                         "report their difference; 0: skip")
    ap.add_argument("--scale-n", type=int, default=2048)
    ap.add_argument("--scale-steps", type=int, default=0,
                    help="instead of the benchmark: the seeded quadrant problem at "
                         "--scale-n^2 cells, mixed against binary64, this many steps")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = _dist_setup()
    if args.scale_steps > 0:
        return run_mixed_at_scale(args) if rank == 0 else 0
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
