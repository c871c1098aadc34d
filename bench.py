#!/usr/bin/env python
"""Benchmark of the blended P2-P1 Stokes hot path on one GB300.

Workload (headline): the spherical shell r in [0.5, 1] (60 macro-tets, radial blending),
refinement level 6 (15,728,640 micro-tets, 63,406,854 velocity + 2,662,530 pressure dofs),
viscosity contrast 1e6 (radial step x plumes x log-normal noise, seed 2), compressible
density d ln rho/dr = -0.3781.  One step = one fused, constrained saddle-point apply
[A B^T; (B+C) 0] (x, p) in FP32 — the operator application that the mixed-precision
solver's Krylov, smoother and residual work is made of.
Metric: GDoF/s = (N_u + N_p) / time per apply / 1e9; and the time to a relative residual of
1e-8 (measured in FP64) of the mixed-precision solve against the plain FP64 GPU solve of the
same problem (assembled buoyancy forcing of a temperature field, compressible density).
The level-5 workload (8,325,576 dofs) is reported beside it under "level5".

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload
(micro-tets of the level-6 shell, evaluated row-sample-wise by oracle/sampled.py, scaled to
the full apply).
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
sys.path.insert(0, ROOT)

METRIC = "P2-P1 Stokes apply GDoF/s; time to 1e-8 residual, mixed vs FP64, 1 GB300"
WORKLOADS = {
    6: "shell-L6-contrast1e6: blended icosahedral shell, level 6, 66,069,384 dofs, FP32 fused constrained Stokes apply",
    5: "shell-L5-contrast1e6: blended icosahedral shell, level 5, 8,325,576 dofs, FP32 fused constrained Stokes apply",
}
# dram__bytes_read.sum + dram__bytes_write.sum of one fused FP32 launch of the default sweep
# variant, per level, from ncu captures of _one launch_ (profiles/ names the command); None
# where no capture of the current kernel exists
MEASURED_DRAM_BYTES = {6: 765305344 + 241406208, 5: 99991552 + 7762688}
DRAM_PROFILE = "profiles/stokes_tile_kernel_fixed_x2_f32_fused_dram.md"
DEFAULT_KERNEL = "stokes_tile_kernel_fixed_x2<float, A|BT|B|C, blended, 128 threads, 4 CTAs/SM>"


def fused_stokes_flops_per_tet():
    """Algorithmic flops of one micro-tet of the fused apply (FMA = 2 flops), counted term by
    term from the per-quadrature-point algebra of the sweep: per tet 60 (nodal sums), per qp
    4 x 300 (position 24, blending Jacobian and K 57, viscosity/pressure at qp 6, lattice
    gradient 36, physical gradient 45, divergence + compressible term 32, stress 25, test side
    45, accumulation 30), final distribution 123."""
    return 60 + 4 * 300 + 123


def algorithmic_bytes(n_p2, n_p1, word):
    """Bytes one fused apply must move at least: u read and y written (3 n_p2 each), p read,
    q written and the nodal viscosity read (n_p1 each); the per-macro geometry is negligible."""
    return word * (6 * n_p2 + 3 * n_p1)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling (20 ms period) with host timestamps; summary()
    uses the samples inside the timed window, else those of the adjacent busy window
    (warm-up through the end of the run), and says which."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
            self.proc = None

    def summary(self):
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), [nm for k, nm in enumerate(names)
                                                            if len(f) > 6 + k and f[6 + k].lower() == "active"]))
            except (ValueError, IndexError):
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1]]
        use, where = (inside, "timed") if inside else (rows, "adjacent busy window")
        reasons = sorted({x for r in use for x in r[3]})
        return {"sm_mhz": statistics.median([r[1] for r in use]), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "window": where}


def aggregate(ms_local, steps, units_per_rank, world, device):
    """Max of the timed region over ranks; whole-job throughput = all ranks' units / that
    time (replicas: every rank processes its own copy of the workload)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / steps
    return ms_per_step, world * units_per_rank / (ms_per_step * 1e-3) / 1e9


def setup_problem(level, device):
    import numpy as np
    import torch
    import paper_2506_04157_gb300 as mfs
    import workloads as W
    ctx = mfs.Context(device)
    mesh = mfs.Mesh(ctx, level)
    prob = mfs.Problem(mesh)
    x1 = mesh.coords(level, p2=False).T
    prob.set_viscosity(torch.tensor(W.viscosity_plumes(x1, seed=2, contrast=1e6), device=f"cuda:{device}"))
    prob.set_density(W.dlnrho_table_compressible())
    inf = mesh.info(level)
    return ctx, mesh, prob, inf


def measure_peaks(ctx):
    """FP32, packed-pair FP32 and FP64 FMA-pipe throughput (mfs_fma_peak: FMA-chain kernels,
    CUDA events, 5 launches of about 0.1-0.2 s each), TFLOP/s."""
    out = {}
    for kind, iters in (("f32", 20000), ("f32x2", 20000), ("f64", 400)):
        tf, ms = ctx.fma_peak(kind, launches=5, iters=iters)
        out[kind] = {"tflops": round(tf, 3), "ms": round(ms, 2)}
    return out


def apply_bench(ctx, prob, inf, level, steps, warmup, world, rank, dev, clk=None):
    """Device-timed fused constrained FP32 applies on rotating input sets (together larger than
    L2), the sweep kernel's own time from CUDA events on the library's stream, the A block alone,
    and the FP64 fused apply (kernel time)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import workloads as W
    nu, npp = 3 * inf.n_p2, inf.n_p1
    dofs = nu + npp
    bytes_per_set = 4 * (2 * nu + 2 * npp)
    l2 = 126 * 2 ** 20
    nsets = max(2, int(np.ceil(2 * l2 / bytes_per_set)))
    sets = []
    for k in range(nsets):
        u = torch.tensor(W.random_field(nu, 100 + k, np.float32), device=dev)
        p = torch.tensor(W.random_field(npp, 200 + k, np.float32), device=dev)
        sets.append((u, p, torch.empty_like(u), torch.empty_like(p)))

    def step(i):
        u, p, yu, yp = sets[i % nsets]
        prob.apply_stokes(level, u, p, yu, yp)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.kernel_time()
    ctx.enable_timing(True)
    torch.cuda.synchronize()
    tw0 = time.time()
    e0.record(stream)
    for i in range(steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    if clk is not None:
        clk.mark(tw0, time.time())
    ctx.enable_timing(False)
    ktot, klaunch = ctx.kernel_time()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ms_per_step, value = aggregate(ms, steps, dofs, world, dev)
    # the A block alone (constrained, the smoother's operator): N_u per sweep-kernel time
    ctx.kernel_time()
    ctx.enable_timing(True)
    for i in range(steps):
        u, p, yu, yp = sets[i % nsets]
        prob.apply_A(level, u, yu, constrained=True)
    torch.cuda.synchronize()
    ctx.enable_timing(False)
    a_tot, a_launch = ctx.kernel_time()
    # FP64 fused apply (plain-precision solver's operator), kernel time
    u64 = sets[0][0].double()
    p64 = sets[0][1].double()
    yu64, yp64 = torch.empty_like(u64), torch.empty_like(p64)
    prob.apply_stokes(level, u64, p64, yu64, yp64)
    torch.cuda.synchronize()
    n64 = 3 if level >= 6 else 10
    ctx.kernel_time()
    ctx.enable_timing(True)
    for _ in range(n64):
        prob.apply_stokes(level, u64, p64, yu64, yp64)
    torch.cuda.synchronize()
    ctx.enable_timing(False)
    d_tot, d_launch = ctx.kernel_time()
    del u64, p64, yu64, yp64
    return {"value": value, "ms_per_step": ms_per_step, "kernel_ms": ktot / max(klaunch, 1),
            "a_ms": a_tot / max(a_launch, 1), "fp64_kernel_ms": d_tot / max(d_launch, 1), "nsets": nsets,
            "bytes_per_set": bytes_per_set, "sets": sets, "dofs": dofs}


def e2e_bench(prob, inf, level, steps, world, dev):
    """The same apply through the public API with host buffers, every step copying its inputs
    (u, p) from pinned host memory to the device and its result (y_u, y_p) back, all inside the
    timed region.  value: the steps streamed through three CUDA streams (host-to-device copies,
    the applies on the problem's stream, device-to-host copies) with two device buffer sets, so
    that step k's apply overlaps step k+1's input copy and step k-1's result copy (events order
    each buffer's reuse); serial_value: the same steps one after another on one stream."""
    import numpy as np
    import torch
    import workloads as W
    nu, npp = 3 * inf.n_p2, inf.n_p1
    dt = torch.float32
    hu = torch.tensor(W.random_field(nu, 7, np.float32)).pin_memory()
    hp = torch.tensor(W.random_field(npp, 8, np.float32)).pin_memory()
    ou = [torch.empty_like(hu).pin_memory() for _ in range(2)]
    op_ = [torch.empty_like(hp).pin_memory() for _ in range(2)]
    du = [torch.empty(nu, dtype=dt, device=dev) for _ in range(2)]
    dp = [torch.empty(npp, dtype=dt, device=dev) for _ in range(2)]
    dyu = [torch.empty_like(du[0]) for _ in range(2)]
    dyp = [torch.empty_like(dp[0]) for _ in range(2)]
    comp = torch.cuda.current_stream()          # the problem's context stream
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    n_e2e = max(3, steps // 2)

    def serial(k):
        b = k % 2
        du[b].copy_(hu, non_blocking=True)
        dp[b].copy_(hp, non_blocking=True)
        prob.apply_stokes(level, du[b], dp[b], dyu[b], dyp[b])
        ou[b].copy_(dyu[b], non_blocking=True)
        op_[b].copy_(dyp[b], non_blocking=True)

    def pipelined(n):
        e_in = [torch.cuda.Event() for _ in range(n)]
        e_done = [torch.cuda.Event() for _ in range(n)]
        e_out = [torch.cuda.Event() for _ in range(n)]
        for k in range(n):
            b = k % 2
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(e_done[k - 2])      # the apply of step k-2 has read du[b], dp[b]
                du[b].copy_(hu, non_blocking=True)
                dp[b].copy_(hp, non_blocking=True)
                e_in[k].record(s_in)
            comp.wait_event(e_in[k])
            if k >= 2:
                comp.wait_event(e_out[k - 2])            # step k-2's result is on the host
            prob.apply_stokes(level, du[b], dp[b], dyu[b], dyp[b])
            e_done[k].record(comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(e_done[k])
                ou[b].copy_(dyu[b], non_blocking=True)
                op_[b].copy_(dyp[b], non_blocking=True)
                e_out[k].record(s_out)
        comp.wait_event(e_out[n - 1])
        comp.wait_stream(s_in)

    for k in range(2):
        serial(k)
    pipelined(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    for k in range(n_e2e):
        serial(k)
    e1.record(comp)
    torch.cuda.synchronize()
    serial_ms = e0.elapsed_time(e1) / n_e2e
    e0.record(comp)
    pipelined(n_e2e)
    e1.record(comp)
    torch.cuda.synchronize()
    pipe_ms = e0.elapsed_time(e1) / n_e2e
    gd = lambda ms: round(world * (nu + npp) / (ms * 1e-3) / 1e9, 3)
    return {"value": gd(pipe_ms), "unit": "GDoF/s",
            "h2d_bytes_per_step": 4 * (nu + npp), "d2h_bytes_per_step": 4 * (nu + npp),
            "steps": n_e2e, "mode": "pipelined: H2D, apply and D2H on three streams, two buffer sets",
            "serial_value": gd(serial_ms)}


def solve_bench(prob, mesh, level, dev, modes):
    """Time to solve: multigrid setup (diag, eigenvalue estimates, coarse inverse) plus the
    solve to relative residual 1e-8 measured in FP64.  Forcing: the assembled buoyancy load
    vector (mfs_rhs_buoyancy) of a temperature field of 8 Gaussian blobs (seed 3) with the
    compressible density profile, gravity -x/|x|, scale 1.  modes: (name, options, timed runs,
    warm-up runs); the reported time is the median of the timed runs."""
    import torch
    nu, npp = 3 * mesh.info(level).n_p2, mesh.info(level).n_p1
    f = buoyancy_forcing(mesh, prob, level, dev)
    g = torch.zeros(npp, dtype=torch.float64, device=dev)
    out = {}
    for name, sopts, reps, warm in modes:
        for _ in range(warm):   # graphs, Krylov storage, caches
            u = torch.zeros(nu, dtype=torch.float64, device=dev)
            p = torch.zeros(npp, dtype=torch.float64, device=dev)
            prob.setup_multigrid(1)
            prob.solve(f, g, u, p, raise_on_error=False, **sopts)
        runs = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prob.setup_multigrid(1)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            u = torch.zeros(nu, dtype=torch.float64, device=dev)
            p = torch.zeros(npp, dtype=torch.float64, device=dev)
            st = prob.solve(f, g, u, p, raise_on_error=False, **sopts)
            torch.cuda.synchronize()
            runs.append((time.perf_counter() - t0, t_setup, st))
        runs.sort(key=lambda r: r[0])
        t_all, t_setup, st = runs[len(runs) // 2]
        out[name] = {"time_to_solve_s": round(t_all, 3), "setup_s": round(t_setup, 3),
                     "runs_s": [round(r[0], 3) for r in runs], "fgmres_iters_runs": [r[2]["fgmres_iters"] for r in runs],
                     "solve_s": round(st["time_ms"] / 1e3, 3), "rel_residual_fp64": st["rel_residual"],
                     "status": st["status"], "fgmres_iters": st["fgmres_iters"],
                     "refinement_steps": st["outer_iters"], "vcycles": st["vcycles"],
                     "parts_s": {"A_block_cg": round(st["time_Ahat_ms"] / 1e3, 3),
                                 "schur_vbfbt": round(st["time_Sinv_ms"] / 1e3, 3),
                                 "of_which_mass_cg": round(st["time_Minv_ms"] / 1e3, 3)}}
        del u, p
    return out


def roofline(level, inf, kern_ms, fp64_ms, peaks):
    """Arithmetic roofline of the fused sweep (FP32 default path and FP64): algorithmic flops
    per launch / kernel time against the FMA-chain peaks measured in this run."""
    flops = fused_stokes_flops_per_tet() * inf.n_tets
    achieved = flops / (kern_ms * 1e-3) / 1e12
    peak = peaks["f32"]["tflops"]
    ach64 = flops / (fp64_ms * 1e-3) / 1e12
    peak64 = peaks["f64"]["tflops"]
    bytes32 = algorithmic_bytes(inf.n_p2, inf.n_p1, 4)
    traffic = MEASURED_DRAM_BYTES.get(level)
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_source": f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one level-{level} launch "
                              f"({DRAM_PROFILE})" if traffic is not None else None,
            "kernel": DEFAULT_KERNEL, "kernel_ms": round(kern_ms, 5), "flops_per_launch": flops,
            "flops_per_tet": fused_stokes_flops_per_tet(),
            "algorithmic_bytes": bytes32, "algorithmic_GB_s": round(bytes32 / (kern_ms * 1e-3) / 1e9, 1),
            "peak_basis": "measured in this run: FP32 FMA-chain kernel (mfs_fma_peak), of measured",
            "fp64": {"bound": "alu", "achieved": round(ach64, 4), "peak": round(peak64, 4), "unit": "TFLOP/s",
                     "frac": round(ach64 / peak64, 4), "kernel": "stokes_tile_kernel<double, A|BT|B|C, blended>",
                     "kernel_ms": round(fp64_ms, 4), "peak_basis": "measured in this run: FP64 FMA-chain kernel"}}


def _optional(fn):
    """Runs an optional part of the bench line (solves, the level-5 lines, the ensemble, the CPU
    baseline); a failure is reported in its place instead of ending the run before the headline
    line is printed."""
    try:
        return fn()
    except Exception as e:   # reported, not fatal: the headline stands
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args, rank, world, device):
    import torch
    torch.cuda.set_device(device)
    dev = f"cuda:{device}"
    level = args.level
    clk = ClockSampler(device).start()
    ctx, mesh, prob, inf = setup_problem(level, device)
    peaks = measure_peaks(ctx)
    ab = apply_bench(ctx, prob, inf, level, args.steps, args.warmup, world, rank, dev, clk)
    e2e = e2e_bench(prob, inf, level, args.steps, world, dev)
    nu, npp = 3 * inf.n_p2, inf.n_p1
    del ab["sets"]
    line = {
        "metric": METRIC, "value": round(ab["value"], 3), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ab["ms_per_step"], 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(level, f"shell-L{level}"), "level": level, "n_tets": inf.n_tets,
                   "n_u": nu, "n_p": npp, "viscosity": "plumes contrast 1e6 seed 2",
                   "density": "compressible, d ln rho/dr = -0.3781",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"{ab['nsets']} rotating input sets of {ab['bytes_per_set'] / 2**20:.1f} MiB (> L2)",
                   "sweep_variant": prob.get_tuning(level)},
        "roofline": roofline(level, inf, ab["kernel_ms"], ab["fp64_kernel_ms"], peaks),
        "e2e": e2e,
        "gpu_launches": int(args.steps * 6),   # per apply: 2 (p sum) + 1 sweep + 2 (q sum) + 1 (mean removal)
        "a_block": {"kernel_ms": round(ab["a_ms"], 5), "gdofs": round(nu / (ab["a_ms"] * 1e-3) / 1e9, 3),
                    "note": "constrained A sweep alone (sweep variant 7: packed pairs, 192 threads, "
                            "3 CTAs/SM), N_u per kernel time"},
        "measured_peaks": peaks,
        "hbm_peak_measured_gbs": read_peaks().get("hbm_gbs"),
    }
    solve = {}
    if args.solve:
        modes = [("mixed_fp64_outer", dict(mixed=2), 2, 1), ("mixed", dict(mixed=1), 1, 0)]
        if args.solve_fp64 and world == 1:
            modes.append(("fp64", dict(mixed=0), 1, 0))
        solve[f"L{level}"] = _optional(lambda: solve_bench(prob, mesh, level, dev, modes))
    del prob, mesh
    torch.cuda.empty_cache()

    def level5():
        # the level-5 workload beside it: apply, roofline, solves, Schur applications
        ctx5, mesh5, prob5, inf5 = setup_problem(5, device)
        ab5 = apply_bench(ctx5, prob5, inf5, 5, args.steps, args.warmup, 1, 0, dev)
        del ab5["sets"]
        out = {"workload": WORKLOADS[5], "value": round(ab5["value"], 3), "unit": "GDoF/s",
               "ms_per_step": round(ab5["ms_per_step"], 5),
               "roofline": roofline(5, inf5, ab5["kernel_ms"], ab5["fp64_kernel_ms"], peaks),
               "a_block": {"kernel_ms": round(ab5["a_ms"], 5),
                           "gdofs": round(3 * inf5.n_p2 / (ab5["a_ms"] * 1e-3) / 1e9, 3)}}
        if args.solve:
            modes5 = [("mixed", dict(mixed=1), args.solve_reps, 1),
                      ("mixed_fp64_outer", dict(mixed=2), args.solve_reps, 1),
                      ("mixed_fp64_outer_adjoint_uzawa", dict(mixed=2, uzawa=2, tol_A=1e-4), args.solve_reps, 1)]
            if args.solve_fp64_l5:
                modes5.append(("fp64", dict(mixed=0), 1, 0))
            solve["L5"] = _optional(lambda: solve_bench(prob5, mesh5, 5, dev, modes5))
            out["schur_apply"] = _optional(lambda: schur_applies(prob5, 5, inf5, dev))
        del prob5, mesh5
        torch.cuda.empty_cache()
        return out

    if level != 5 and world == 1 and not args.no_level5:
        line["level5"] = _optional(level5)
    clk.stop()
    if rank != 0:
        return None
    if solve:
        line["time_to_solve"] = solve
    line["clocks"] = clk.summary()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _optional(lambda: cpu_baseline(level, budget_s=args.cpu_seconds))
    if world == 1 and args.solve and not args.no_ensemble:
        line["ensemble"] = _optional(lambda: ensemble_bench(device, sequential=args.ensemble))
    return line


def ensemble_bench(device, n_members=64, n_streams=8, sequential=False):
    """The ensemble workload: n_members shells with refinement levels drawn from {3, 4, 5},
    log-uniform viscosity contrast in [1e4, 1e6] (plumes, seeds 100 + i), compressible
    density, buoyancy forcing from a seeded temperature field per member; FP32 applies in FP64
    refinement (mixed = 1) to 1e-8, at most 1000 FGMRES iterations.  Time to solve all members (wall clock, device synchronized
    before and after): one member after another (one host thread) and concurrently
    (mfs_solve_concurrent, one host thread per stream), from zero initial guesses each time.
    The one-after-another run only when `sequential`."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2506_04157_gb300 as mfs
    dev = f"cuda:{device}"
    rng = np.random.default_rng(3)
    levels = rng.integers(3, 6, size=n_members)
    contrasts = 10.0 ** rng.uniform(4.0, 6.0, size=n_members)
    ens = mfs.Ensemble(levels, n_streams=n_streams, device=device)
    fs, gs = [], []
    t0 = time.perf_counter()
    for i, (l, c) in enumerate(zip(levels, contrasts)):
        l = int(l)
        P = ens.problems[i]
        x1 = P.mesh.coords(l, p2=False).T
        P.set_viscosity(torch.tensor(W.viscosity_plumes(x1, 100 + i, float(c)), device=dev))
        P.set_density(W.dlnrho_table_compressible())
        P.setup_multigrid(1)
        T = torch.tensor(W.temperature_blobs(P.mesh.coords(l).T, 500 + i), device=dev)
        f = torch.empty(3 * T.numel(), dtype=torch.float64, device=dev)
        P.rhs_buoyancy(T, f, scale=1.0)
        fs.append(f)
        gs.append(torch.zeros(P._sizes(l)[1], dtype=torch.float64, device=dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = {"members": n_members, "levels": {str(l): int((levels == l).sum()) for l in (3, 4, 5)},
           "dofs": int(sum(sum(P._sizes(int(l))) for P, l in zip(ens.problems, levels))),
           "streams": n_streams, "mixed": 1, "setup_s": round(setup_s, 3)}
    runs = (("sequential", 1), ("concurrent", 0)) if sequential else (("concurrent", 0),)
    for name, nt in runs:
        us = [torch.zeros_like(f) for f in fs]
        ps = [torch.zeros_like(g) for g in gs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = ens.solve(fs, gs, us, ps, n_threads=nt, raise_on_error=False, mixed=1, max_iters=1000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = [st["fgmres_iters"] for st in stats]
        out[name] = {"time_to_solve_s": round(dt, 3), "threads": 1 if nt == 1 else min(n_streams, n_members),
                     "fgmres_iters_min_max": [int(min(its)), int(max(its))],
                     "converged": int(sum(st["rel_residual"] <= 1e-8 for st in stats)),
                     "max_rel_residual_fp64": max(st["rel_residual"] for st in stats)}
    if sequential:
        out["speedup"] = round(out["sequential"]["time_to_solve_s"] / out["concurrent"]["time_to_solve_s"], 3)
    out["note"] = ("each member's solve reaches 1e-8 measured in FP64; the concurrent run overlaps the "
                   "members of different streams (mfs_solve_concurrent)")
    del ens
    torch.cuda.empty_cache()
    return out


def buoyancy_forcing(mesh, prob, level, dev):
    """f = int rho(r) T (x/|x|) . phi on the finest level (mfs_rhs_buoyancy), T the nodal P2
    temperature of 8 Gaussian blobs (seed 3)."""
    import torch
    import workloads as W
    T = torch.tensor(W.temperature_blobs(mesh.coords(level).T, 3), device=dev)
    f = torch.empty(3 * T.numel(), dtype=torch.float64, device=dev)
    prob.rhs_buoyancy(T, f, scale=1.0)
    return f


def schur_applies(prob, level, inf, dev):
    """One application of each Schur approximation (FP32, the solver's tolerances; wall time
    including the host synchronisations of their inner CGs, median of 3 after a warm-up) and
    the weighted BFBT's K_{1/sqrt(eta)} sweep alone (CUDA events, 20 launches after 3): its
    algorithmic bytes are the 6 FP32 element entries per micro-tet plus the P1 input and
    output vectors."""
    import numpy as np
    import torch
    import paper_2506_04157_gb300 as mfs
    import workloads as W
    npp = inf.n_p1
    r = torch.tensor(W.random_field(npp, 41, np.float32), device=dev)
    r -= r.mean()
    z = torch.empty_like(r)
    out = {}
    try:
        times = {}
        for name, schur in (("vbfbt", 0), ("mass", 1), ("wbfbt", 3)):
            prob.apply_schur(r, z, schur=schur)
            ts, st = [], None
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = prob.apply_schur(r, z, schur=schur)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            times[name] = {"ms": round(1e3 * sorted(ts)[1], 3), "cg_X_iters": st["cg_X_iters"],
                           "cg_M_iters": st["cg_M_iters"]}
        out["fp32_apply"] = times
        y = torch.empty_like(r)
        for _ in range(3):
            prob.apply_poisson(level, 1.0, r, y)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            prob.apply_poisson(level, 1.0, r, y)
        e1.record(stream)
        torch.cuda.synchronize()
        k_ms = e0.elapsed_time(e1) / 20
        nbytes = 24 * inf.n_tets + 8 * npp
        gbs = nbytes / (k_ms * 1e-3) / 1e9
        hbm = read_peaks().get("hbm_gbs")
        out["K_sweep"] = {"ms": round(k_ms, 5), "bytes": nbytes, "GB_s": round(gbs, 1),
                          "frac_of_measured_hbm": round(gbs / hbm, 3) if hbm else None,
                          "note": "K_{1/sqrt(eta)} apply (memset + sweep), FP32"}
    except mfs.MfsError as e:
        out["error"] = str(e)
    return out


def profile_solve(level):
    """A window of solver work between cudaProfilerStart/Stop (everything before it warms
    up the captured graphs): the launch list of the V-cycles and one preconditioned FGMRES
    iteration."""
    import numpy as np
    import torch
    import workloads as W
    ctx, mesh, prob, inf = setup_problem(level, 0)
    prob.setup_multigrid(1)
    u = torch.tensor(W.random_field(3 * inf.n_p2, 5, np.float32), device="cuda")
    y = torch.empty_like(u)
    f = buoyancy_forcing(mesh, prob, level, "cuda")
    g = torch.zeros(inf.n_p1, dtype=torch.float64, device="cuda")
    uu = torch.zeros(3 * inf.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(g)
    for _ in range(3):
        prob.vcycle(level, u, y, 3, 2)
        prob.vcycle(level, u, y, 1, 1)
    prob.solve(f, g, uu, p, raise_on_error=False, mixed=1, max_iters=1, max_outer=1)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    prob.vcycle(level, u, y, 3, 2)
    prob.vcycle(level, u, y, 1, 1)
    uu.zero_()
    p.zero_()
    st = prob.solve(f, g, uu, p, raise_on_error=False, mixed=1, max_iters=1, max_outer=1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_window": "vcycle(3,2) + vcycle(1,1) + 1 FGMRES iteration", "level": level,
                      "vcycles": st["vcycles"], "status": st["status"]}))


_ORACLE_WORKLOADS = {}


def _oracle_workload(level):
    """The oracle side of the bench workload, without building the level's global element
    arrays: the per-macro micro-tet lattice (oracle/sampled.py), the plume viscosity at the
    blended vertex positions, and random inputs (built once; not timed)."""
    if level not in _ORACLE_WORKLOADS:
        import workloads as W
        from oracle.mesh import MacroMesh, lattice_nodes
        from oracle.sampled import MacroRows
        mesh = MacroMesh()
        R = MacroRows(mesh, level)
        X1, _, pr1 = lattice_nodes(mesh, 2 ** level)
        eta = W.viscosity_plumes(mesh.blend(X1, pr1), seed=2, contrast=1e6)
        _ORACLE_WORKLOADS[level] = (R, eta, W.random_field(3 * R.n_p2, 1), W.random_field(R.n_p1, 2))
    return _ORACLE_WORKLOADS[level]


def _sample_apply(level, budget_s, seed, chunk=4096):
    """(micro-tets swept, seconds): the FP64 oracle's fused element apply (A u + B^T p,
    (B + C) u; oracle/sampled.py MacroRows.contributions) on random chunks of micro-tets of
    random macros until budget_s of CPU time is used."""
    import numpy as np
    import workloads as W
    R, eta, u, p = _oracle_workload(level)
    ntet = R.kt.shape[0]
    rng = np.random.default_rng(seed)
    done, t_used = 0, 0.0
    dl = W.dlnrho_table_compressible()
    while t_used < budget_s:
        m = int(rng.integers(0, 60))
        sel = np.sort(rng.choice(ntet, size=min(chunk, ntet), replace=False))
        t0 = time.perf_counter()
        R.contributions(m, sel, eta, dl, u, p)
        t_used += time.perf_counter() - t0
        done += len(sel)
    return done, t_used


def cpu_baseline(level, budget_s=12.0):
    """The FP64 oracle's fused apply on a bounded sample of micro-tets of the same workload,
    one core, scaled to the full level (GDoF/s)."""
    R, _, _, _ = _oracle_workload(level)
    done, t_used = _sample_apply(level, budget_s, 0)
    n_tets = 60 * R.kt.shape[0]
    t_full = t_used * n_tets / done
    dofs = 3 * R.n_p2 + R.n_p1
    return {"value": round(dofs / t_full / 1e9, 7), "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} of {n_tets} micro-tets of the level-{level} shell (random chunks of 4096 in random "
                      f"macros), {t_used:.1f} s, scaled to one full apply",
            "dofs_per_apply": dofs}


def _sample_worker(level, budget_s, seed):
    """One process of the all-cores CPU baseline: (micro-tets swept, seconds)."""
    return _sample_apply(level, budget_s, seed)


def cpu_baseline_all_cores(level, budget_s=3.0, max_procs=16):
    """The same sampled oracle apply in one process per host core (spawned; each builds its
    own copy of the workload), throughput summed over the processes (GDoF/s), or None."""
    import multiprocessing as mp
    n = max(1, min(os.cpu_count() or 1, max_procs))
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.starmap(_sample_worker, [(level, budget_s, 1000 + k) for k in range(n)])
    except Exception as e:   # reported, not fatal: the one-core baseline stands
        return {"error": f"{type(e).__name__}: {e}"}
    R, _, _, _ = _oracle_workload(level)
    tets_per_s = sum(d / t for d, t in res)
    dofs = 3 * R.n_p2 + R.n_p1
    return {"value": round(dofs * tets_per_s / (60 * R.kt.shape[0]) / 1e9, 7), "unit": "GDoF/s", "cores": n,
            "kind": "oracle", "sample": f"{n} processes x {budget_s:.0f} s of random 4096-tet chunks"}


def oracle_levels(budget_s=3.0):
    """The oracle at the configured sizes it can run here: the fused apply at levels 2-4 (full
    sweeps, level 4 sampled within budget_s) and the solve to 1e-8 of the level-2 shell
    (config 1: radial viscosity, d ln rho/dr = -1; symmetric Uzawa, V-cycle BFBT, FGMRES)."""
    import numpy as np
    import workloads as W
    from oracle.mesh import MacroMesh, Level
    from oracle.fem import stokes_apply_elements
    from oracle.solver import Hierarchy, StokesOracle
    out = {}
    for lvl in (2, 3, 4):
        L = Level(MacroMesh(), lvl)
        eta = W.viscosity_plumes(L.p1_x, seed=2, contrast=1e6)
        u, p = W.random_field(3 * L.n_p2, 1), W.random_field(L.n_p1, 2)
        ntet = L.tet_p2.shape[0]
        sel = np.arange(ntet) if lvl < 4 else np.arange(min(ntet, 16384))
        t0 = time.perf_counter()
        stokes_apply_elements(L, eta, W.dlnrho_table_compressible(), u, p, sel)
        dt = (time.perf_counter() - t0) * ntet / len(sel)
        out[f"apply_L{lvl}_gdofs"] = round((3 * L.n_p2 + L.n_p1) / dt / 1e9, 7)
    mesh = MacroMesh()
    L2 = Level(mesh, 2)
    H = Hierarchy(mesh, 2, W.viscosity_radial(L2.p1_x), dlnrho_table=W.dlnrho_table_config1())
    f = W.random_field(3 * L2.n_p2, 3)
    t0 = time.perf_counter()
    _, _, it, _ = StokesOracle(H).solve(f, np.zeros(L2.n_p1), np.zeros(3 * L2.n_p2), np.zeros(L2.n_p1), rtol=1e-8)
    out["solve_L2_s"] = round(time.perf_counter() - t0, 2)
    out["solve_L2_fgmres_iters"] = int(it)
    out["cores"] = 1
    return out


def compare_preconditioners(level, max_iters=200):
    """The block preconditioners and Schur approximations of Sec. 5.2 on the same workload and
    forcing as the bench's solves (FP64 outer FGMRES around the FP32 preconditioner, mixed = 2;
    tol_A 1e-4 for the one-sided Uzawa steps): FGMRES iterations, time, reached residual."""
    import torch
    ctx, mesh, prob, inf = setup_problem(level, 0)
    dev = "cuda:0"
    f = buoyancy_forcing(mesh, prob, level, dev)
    g = torch.zeros(inf.n_p1, dtype=torch.float64, device=dev)
    out = {}
    for sname, schur in (("vbfbt", 0), ("mass", 1), ("diagA_bfbt", 2), ("wbfbt_consistent", 3)):
        for uname, uzawa in (("symmetric", 0), ("inexact", 1), ("adjoint_inexact", 2)):
            opts = dict(mixed=2, schur=schur, uzawa=uzawa, max_iters=max_iters)
            if uzawa:
                opts["tol_A"] = 1e-4
            prob.setup_multigrid(1)
            u = torch.zeros(3 * inf.n_p2, dtype=torch.float64, device=dev)
            p = torch.zeros(inf.n_p1, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = prob.solve(f, g, u, p, raise_on_error=False, **opts)
            torch.cuda.synchronize()
            out[f"{sname}/{uname}"] = {"fgmres_iters": st["fgmres_iters"], "time_s": round(time.perf_counter() - t0, 2),
                                       "rel_residual": st["rel_residual"], "status": st["status"]}
            print(json.dumps({f"{sname}/{uname}": out[f"{sname}/{uname}"]}), flush=True)
    print(json.dumps({"compare_preconditioners": out, "level": level}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # each step: one bounded sample of the workload (random micro-tets of the level, their
    # fused element apply); value = the sample's dofs-equivalent throughput, ms_per_step = the
    # sample's measured duration
    rates, step_ms = [], []
    cb = None
    _oracle_workload(args.level)   # built once, outside the timed samples
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(args.level, budget_s=max(0.5, args.cpu_seconds / max(1, args.steps)))
        if i >= args.warmup:
            rates.append(cb["value"])
            step_ms.append(1e3 * (time.perf_counter() - t0))
    v = statistics.median(rates)
    cb["value"] = v
    ms_per_step = statistics.median(step_ms)
    return {"metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOADS.get(args.level, f"shell-L{args.level}"), "level": args.level},
            "cpu_baseline": cb,
            "oracle_levels": oracle_levels(),
            "cpu_baseline_all_cores": cpu_baseline_all_cores(args.level),
            "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=6)
    ap.add_argument("--no-level5", action="store_true", help="skip the level-5 lines beside the headline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve", dest="solve", action="store_true", default=True,
                    help="also time the mixed-precision solve to 1e-8 (default)")
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--solve-fp64", dest="solve_fp64", action="store_true", default=True,
                    help="also time the plain FP64 GPU solve of the same problem (default at 1 GPU)")
    ap.add_argument("--no-solve-fp64", dest="solve_fp64", action="store_false")
    ap.add_argument("--solve-fp64-l5", action="store_true", help="also the plain FP64 solve at level 5")
    ap.add_argument("--solve-reps", type=int, default=3, help="level-5 mixed-precision solves (median reported)")
    ap.add_argument("--compare-preconditioners", action="store_true",
                    help="only the Uzawa x Schur comparison of the solver on the --level workload")
    ap.add_argument("--ensemble", action="store_true",
                    help="the 64-member ensemble (levels 3-5) also solved one member after another")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-member ensemble solve")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiler window only (cudaProfilerStart/Stop): one V-cycle (3,2), one V-cycle "
                         "(1,1) and a solve capped at one FGMRES iteration, for ncu --profile-from-start off")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile_solve:
        profile_solve(args.level)
        return
    if args.compare_preconditioners:
        compare_preconditioners(args.level)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        import torch
        import torch.distributed as dist
        if world > 1:
            dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        line = run_ours(args, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
