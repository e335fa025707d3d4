"""Benchmark of the SRJ hot path on GB300 (one JSON line on stdout).

Workload (default): 2-D Dirichlet Poisson, 4096 x 4096 interior points, f a
seeded N(0,1) field smoothed by a 5x5 box mean, Dirichlet data from a seeded
cubic polynomial, optimal P = 10 SRJ schedule for this grid, FP32 sweeps inside
FP64 defect correction, tolerance 1e-10 on the relative L2 residual.

One step = one full solve from the initial guess to the tolerance (all sweeps,
residual checks and corrections).  value = Gupdates/s = sweeps x interior
points / step time; time-to-tolerance is reported beside it, with the plain
FP64 SRJ on the same grid as the comparator.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl srj|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (--ref-sweeps sweeps of the full grid per step, ~1 s) on one host
core; the main line's cpu_baseline is the same oracle on --cpu-sweeps sweeps
(~9 s).
Multi-GPU (torchrun): every rank solves its own replica of the workload
(independent problems, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 residual & Gupdates/s vs plain FP64 SRJ on same GB300; % HBM peak"
N = 4096
P = 10
TOL = 1e-10
SEED_F = 2
MAX_CYCLES = 200
# DRAM bytes (read + write) per launch from one ncu capture of the kernel at
# this grid size (warm cache, --cache-control none; the second captured launch,
# whose writes are its own output only), keyed by (kernel, n).  Entries are
# removed when the kernel changes.
MEASURED_TRAFFIC = {("k_sweep_f32_tb<8,8>", 4096): 201_138_176}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="srj", choices=["srj", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--P", type=int, default=P)
    ap.add_argument("--fp64-cycles", type=int, default=0,
                    help="cycles of the plain FP64 comparator to time (0 = run it to tolerance)")
    ap.add_argument("--cpu-sweeps", type=int, default=256,
                    help="oracle sweeps in the main line's CPU baseline sample (~9 s on one core at 4096^2)")
    ap.add_argument("--ref-sweeps", type=int, default=32,
                    help="oracle sweeps per step of --impl reference (~1 s per step at 4096^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 3-D 512^3 and batched secondary measurements")
    ap.add_argument("--kernel-case", choices=["f32", "f64", "sph", "sphmix", "batch"], default=None,
                    help="profiling aid: run --count sweeps of one precision on an --n x --n grid "
                         "(plain Jacobi weight) through srj_steps, or (batch) one untimed and one timed "
                         "solve of the batched workload, and exit; prints no JSON")
    ap.add_argument("--count", type=int, default=4)
    ap.add_argument("--ndim", type=int, default=2, choices=[2, 3], help="kernel-case: grid dimension (n^ndim points)")
    ap.add_argument("--T", type=int, default=None,
                    help="kernel-case f32 / batch: temporal depth (default: the plan's / the depth tuner's)")
    ap.add_argument("--variant", type=int, default=None, help="kernel-case f32: blocked sweep variant (0..3)")
    return ap.parse_args()


def run_kernel_case(args):
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    n = args.n
    torch.cuda.set_device(0)
    dims = (n,) * args.ndim
    if args.kernel_case == "batch":
        res = batched_workload(torch.cuda.current_stream(), depth=args.T)
        print("kernel case batch:", res)
        return 0
    if args.kernel_case == "sphmix":  # one mixed-precision cycle of the Sect. 5.2 test (blocked FP32 sweeps)
        from paper_1511_04292_gb300 import spherical as sp
        b_h, u0_h = W.spherical_problem_2d(n, 5)
        row = srj.schedules.lookup(2, n, 10) if (2, n, 10) in srj.schedules.available() else \
            srj.schedules.lookup(2, 1024, 10)
        splan = sp.SphericalPlan((n, n), row["omega"], row["q"], row["order"], precision="mixed")
        splan.solve(torch.from_numpy(b_h).cuda(), torch.from_numpy(u0_h).cuda(), 1e-30, 1, check_status=False)
        torch.cuda.synchronize()
        print("kernel case sphmix n=%d done" % n)
        return 0
    if args.kernel_case == "sph":
        from paper_1511_04292_gb300 import spherical as sp
        splan = sp.SphericalPlan(dims, [1.0], [1])
        f = torch.from_numpy(W.random_field(dims, 1)).cuda()
        u = torch.from_numpy(W.random_field(dims, 2)).cuda()
        splan.steps(f, u, 0, args.count)
        torch.cuda.synchronize()
        print("kernel case sph n=%d^%d count=%d done" % (n, args.ndim, args.count))
        return 0
    plan = srj.Plan(dims, 1.0 / (n + 1), [1.0], [1], None, "mixed" if args.kernel_case == "f32" else "fp64")
    if args.T is not None:
        plan.set_temporal_depth(args.T)
    if args.variant is not None:
        plan.set_sweep_variant(args.variant)
    f = torch.from_numpy(W.random_field(dims, 1)).cuda()
    u = torch.from_numpy(W.random_field(dims, 2)).cuda()
    plan.steps(f, u, 0, args.count)
    torch.cuda.synchronize()
    print("kernel case %s n=%d^%d count=%d done" % (args.kernel_case, n, args.ndim, args.count))
    return 0


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        try:
            rows = open(self.path).read().strip().splitlines()
        except OSError:
            rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in rows:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if self.path:
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(args):
    return {"workload": "2d_poisson_%dx%d_srj_P%d_mixed_fp32_sweeps_fp64_correction" % (args.n, args.n, args.P),
            "grid": [args.n, args.n], "stencil": "5-point", "levels_P": args.P, "tol": TOL,
            "rhs": "seeded N(0,1) field, 5x5 box mean (seed %d); Dirichlet data: seeded cubic polynomial" % SEED_F,
            "step": "one full solve from u0 to tolerance",
            "l2": "flushed between timed steps (256 MiB write); per-sweep working set ~134 MB ~ L2 size"}


def _timed(stream, fn):
    """(result, ms) of fn() between two CUDA events on `stream` (synchronised)."""
    import torch
    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream); r = fn(); b.record(stream)
    torch.cuda.synchronize()
    return r, a.elapsed_time(b)


def _hbm_roofline(kernel, bytes_per_launch, launch_us, peaks, note=None):
    gbs = bytes_per_launch / (launch_us * 1e-6) / 1e9
    out = {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": gbs / peaks["hbm_gbs"], "traffic": None, "algorithmic_bytes_per_launch": bytes_per_launch,
           "avg_launch_us": launch_us}
    if note:
        out["note"] = note
    return out


# Relative tolerance of the adjoint solve of the gradient line: its right-hand
# side u - u_t is smooth, so its FP64 floor relative to that right-hand side is
# ~unit roundoff x cond(A) ~ 2e-10 at 2048^2 (the forward solve's is ~1e-12).
ADJOINT_TOL = 1e-9

# FP64 sweep roof: GB300 issues 2 FP64 instructions per clock per SM (1.25
# TFLOP/s counting an FMA as 2 flops).  A 2-D step is 8 FP64 instructions per
# update in the oracle's order (4 adds, 2 multiplies, a subtract, an add) and 6
# with fused multiply-adds (4 adds, 2 FMAs), so the ALU roof is
# 2 x 152 x 2.07e9 / 8 or / 6 updates per second.
FP64_OPS_PER_UPDATE = {"fp64": 8, "fp64fma": 6}


def _fp64_alu_roofline(kernel, updates, seconds, sm_count, sm_mhz, form="fp64fma"):
    peak = 2.0 * sm_count * sm_mhz * 1e6 / 1e12  # T FP64 instructions per second (an FMA counts once)
    ops = FP64_OPS_PER_UPDATE[form]
    ach = ops * updates / seconds / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "peak_source": "derived: 2 FP64 instructions/clock/SM x %d SMs x %.0f MHz" % (sm_count, sm_mhz),
            "ops_per_update": ops, "ops": "FP64 instructions (an FMA counts once)"}


def config1_workload(stream, peaks):
    """128^2 interior, FP64, manufactured solution, P = 5, tol 1e-10: GPU time to
    tolerance (FP64 and mixed) and the oracle run to convergence on one core."""
    import numpy as np
    import torch
    import oracle
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    n = 128
    dims = (n, n)
    f_h, _, u0_h = W.manufactured_2d(n)
    f = torch.from_numpy(f_h).cuda(); u0 = torch.from_numpy(u0_h).cuda(); u = torch.empty_like(u0)
    res = {}
    for prec in ("fp64", "mixed"):
        plan = srj.Plan.from_table(dims, 5, prec)
        for _ in range(3):
            u.copy_(u0); plan.solve(f, u, 1e-10, 2000)
        u.copy_(u0)
        st, ms = _timed(stream, lambda: plan.solve(f, u, 1e-10, 2000))
        res[prec] = {"time_to_tol_s": ms / 1e3, "cycles": st["cycles"], "sweeps": st["sweeps"],
                     "gupdates_per_s": st["sweeps"] * n * n / (ms / 1e3) / 1e9, "final_rel_residual": st["rel_res"]}
        if prec == "fp64":
            M = plan.info()["M"]
            launch_us = st["sweep_ms"] * 1e3 / st["sweeps"]
            res[prec]["roofline"] = _hbm_roofline(
                "k_sweep_f64<2>", 24 * n * n, launch_us, peaks,
                "403 KB working set: L2-resident and launch-latency bound, far from any HBM roof")
            res[prec]["sweep_kernel"] = "k_sweep_f64<2> (one FP64 step per launch, %d launches per cycle graph)" % M
    row = srj.schedules.lookup(2, n, 5)
    seq = oracle.omega_sequence(row["omega"], row["order"])
    oracle.build()
    uo = u0_h.copy()
    t0 = time.perf_counter()
    so = oracle.solve(dims, 1.0 / (n + 1), seq, f_h, uo, 1e-10, 2000)
    dt = time.perf_counter() - t0
    return {"2d_poisson_128x128_P5_fp64_manufactured_tol1e-10": dict(
        res["fp64"], mixed=res["mixed"],
        cpu_baseline={"value": dt, "unit": "s to tol (measured)", "cores": 1, "kind": "oracle",
                      "sample": "full solve to 1e-10: %d cycles, %d sweeps, rel residual %.3g" %
                                (so["cycles"], so["sweeps"], so["rel"])},
        speedup_gpu_fp64_vs_oracle=dt / res["fp64"]["time_to_tol_s"])}


def workload_3d(stream, peaks):
    """512^3, 8 Gaussian blobs, P = 12, tol 1e-9: mixed solve (blocked FP32
    sweeps at the autotuner's depth) and the plain FP64 SRJ comparator (one
    cycle timed, times the cycles the mixed solve needed: the cycle map is the
    same in exact arithmetic)."""
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    n = 512
    f_h, u0_h = W.gaussian_blobs_3d(n, 3)
    f = torch.from_numpy(f_h).cuda(); u0 = torch.from_numpy(u0_h).cuda(); u = torch.empty_like(u0)
    del f_h, u0_h
    plan = srj.Plan.from_table((n, n, n), 12, "mixed")
    T, tuned_us = plan.autotune()
    M = plan.info()["M"]
    u.copy_(u0); plan.solve(f, u, 1e-9, 200)  # warm-up
    u.copy_(u0)
    st, ms = _timed(stream, lambda: plan.solve(f, u, 1e-9, 200))
    launches = st["cycles"] * -(-M // T)
    out = {"time_to_tol_s": ms / 1e3, "gupdates_per_s": st["sweeps"] * n ** 3 / (ms / 1e3) / 1e9,
           "cycles": st["cycles"], "final_rel_residual": st["rel_res"], "temporal_depth": T,
           "autotune_us_per_step": tuned_us,
           "sweep_kernel": "k_sweep3_f32_tb<%d> (%d steps per launch)" % (T, T) if T > 1 else "k_sweep_f32<3>",
           "roofline": _hbm_roofline("k_sweep3_f32_tb<%d>" % T if T > 1 else "k_sweep_f32<3>", 12 * n ** 3,
                                     st["sweep_ms"] * 1e3 / launches, peaks,
                                     "algorithmic bytes of one launch (T steps per HBM round trip); with T = 3 the "
                                     "kernel is bound by instruction issue (69% issue-active), with T = 2 by its HBM "
                                     "stream" if T > 1 else None)}
    del plan
    torch.cuda.empty_cache()
    p64 = srj.Plan.from_table((n, n, n), 12, "fp64fma")
    u.copy_(u0)
    st64, ms64 = _timed(stream, lambda: p64.solve(f, u, 0.0, 1, raise_on_fail=False))
    cyc_ms = st64["sweep_ms"]
    t64 = (ms64 - cyc_ms) / 1e3 + cyc_ms / 1e3 * st["cycles"]
    out["fp64_comparator"] = {
        "time_to_tol_s": t64, "kind": "extrapolated: one FP64 cycle timed (%.0f ms), times the %d cycles of the "
                                      "mixed solve, plus the measured set-up" % (cyc_ms, st["cycles"]),
        "gupdates_per_s": M * n ** 3 / (cyc_ms / 1e3) / 1e9, "sweep_kernel": "k_sweep_f64<3,fma>"}
    out["speedup_vs_fp64_time_to_tol"] = t64 / (ms / 1e3)
    del p64, f, u0, u
    torch.cuda.empty_cache()
    return {"3d_poisson_512^3_P12_mixed_tol1e-9": out}


def spherical_workload(stream, peaks):
    """Sect. 5.2 operator (axisymmetric r-theta), 1024^2, P = 10, tol 1e-10:
    mixed (blocked FP32 cycles) with FP64 beside it."""
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    from paper_1511_04292_gb300 import spherical as sp
    ns = 1024
    b_h, u0_h = W.spherical_problem_2d(ns, 5)
    bs = torch.from_numpy(b_h).cuda(); us0 = torch.from_numpy(u0_h).cuda(); us = torch.empty_like(us0)
    row = srj.schedules.lookup(2, ns, 10)
    act = (ns - 1) * ns
    res = {}
    for prec in ("mixed", "fp64"):
        splan = sp.SphericalPlan((ns, ns), row["omega"], row["q"], row["order"], precision=prec)
        us.copy_(us0); splan.solve(bs, us, 1e-10, 400)  # warm-up
        us.copy_(us0)
        st, ms = _timed(stream, lambda: splan.solve(bs, us, 1e-10, 400))
        res[prec] = dict(time_to_tol_s=ms / 1e3, gupdates_per_s=st["sweeps"] * act / (ms / 1e3) / 1e9,
                         cycles=st["cycles"], final_rel_residual=st["rel_res"])
        if prec == "mixed":
            T = splan.temporal_depth()
            launches = st["cycles"] * -(-len(row["order"]) // T)
            res[prec]["temporal_depth"] = T
            res[prec]["sweep_kernel"] = (f"k_sph_tb<{T}> ({T} FP32 steps per launch, FP64 correction)" if T > 1
                                         else "k_sph_sweep_f32<2> (FP32 cycles, FP64 correction)")
            res[prec]["roofline"] = _hbm_roofline(
                f"k_sph_tb<{T}>" if T > 1 else "k_sph_sweep_f32<2>", 12 * act, st["sweep_ms"] * 1e3 / launches, peaks,
                "12.6 MB working set: L2-resident at this size, bound by FP32 issue (ncu summary)")
        del splan
    del bs, us0, us
    torch.cuda.empty_cache()
    return {"spherical_2d_1024x1024_P10_mixed_tol1e-10": dict(
        res["mixed"], fp64_comparator=dict(res["fp64"], sweep_kernel="k_sph_sweep<2> (FP64)"),
        speedup_vs_fp64_time_to_tol=res["fp64"]["time_to_tol_s"] / res["mixed"]["time_to_tol_s"])}


def adjoint_workload(stream, peaks, sm_count, sm_mhz):
    """Gradient of L = 1/2 ||u - u_t||^2 w.r.t. f and the Dirichlet data, 2048^2,
    FP64, P = 10: forward solve and adjoint solve through the autograd Function."""
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    from paper_1511_04292_gb300.autograd import srj_solve
    na = 2048
    fa_h, ga_h = W.random_smooth_problem_2d(na, 6)
    ta = torch.from_numpy(W.smooth_target_2d(na, 7)).cuda()
    fa = torch.from_numpy(fa_h).cuda().requires_grad_(True)
    ga = torch.from_numpy(ga_h).cuda().requires_grad_(True)
    aplan = srj.Plan.from_table((na, na), 10, "fp64fma")
    # untimed: the same expression on a 64^2 problem loads PyTorch's own kernels (loss, autograd)
    wplan = srj.Plan.from_table((64, 64), 5, "fp64fma")
    wf = torch.zeros(66, 66, dtype=torch.float64, device="cuda", requires_grad=True)
    wg = torch.zeros(66, 66, dtype=torch.float64, device="cuda", requires_grad=True)
    (0.5 * ((srj_solve(wf, wg, wplan, 1e-10, 50) - ta[:66, :66])[1:-1, 1:-1] ** 2).sum()).backward()
    del wplan, wf, wg
    torch.cuda.synchronize()
    ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    ea.record(stream)
    ua = srj_solve(fa, ga, aplan, 1e-10, 400, adjoint_tol=ADJOINT_TOL)
    loss = 0.5 * ((ua - ta)[1:-1, 1:-1] ** 2).sum()
    eb.record(stream)
    loss.backward()
    ec.record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = ea.elapsed_time(eb), eb.elapsed_time(ec)
    fstats = ua.grad_fn.stats
    bstats = ua.grad_fn.adjoint_stats
    upd = (fstats["sweeps"] + bstats["sweeps"]) * na * na
    sweep_s = (fstats["sweep_ms"] + bstats["sweep_ms"]) / 1e3
    out = {"forward_s": fwd_ms / 1e3, "backward_s": bwd_ms / 1e3, "time_s": (fwd_ms + bwd_ms) / 1e3,
           "gupdates_per_s": upd / ((fwd_ms + bwd_ms) / 1e3) / 1e9, "forward_cycles": fstats["cycles"],
           "adjoint_cycles": bstats["cycles"], "forward_rel_residual": fstats["rel_res"],
           "adjoint_rel_residual": bstats["rel_res"], "adjoint_tol": ua.grad_fn.adjoint_tol,
           "sweep_kernel": "k_sweep_f64<2,fma> (FP64 steps with fused multiply-adds)",
           "roofline": _fp64_alu_roofline("k_sweep_f64<2,fma>", upd, sweep_s, sm_count, sm_mhz)}
    del fa, ga, ta, ua, loss, aplan
    torch.cuda.empty_cache()
    return {"adjoint_2d_2048x2048_P10_fp64_tol1e-10": out}


def large_grid_workload(stream, peaks, T, variant, steps=512):
    """Throughput at 2^15 points per dimension (32768^2, up to ~30 GB on the
    device).  Per-step times come from (time of 2K steps - time of K steps) / K,
    which removes the FP64 <-> FP32 conversions srj_steps does around its sweeps.

    FP64: the optimal P = 10 scheme of this grid from the library's planner and
    cycle order; time to tolerance is an estimate, M steps per cycle x the cycle
    count the worst eigenmode needs (the plan's max cycle factor) x the per-step
    time.  Mixed precision: the optimal scheme's largest weight (~1.6e8) makes
    one step amplify the kappa ~ 2 modes by |1 - 2 omega_1| ~ 3e8 > 1 / eps_32,
    and the plan rejects its cycle order (modelled FP32 cycle noise above the
    limit); the FP32 blocked sweep is timed on this grid with the scheme of the
    4096^2 grid instead (coarser-grid parameters remain convergent on finer
    grids, Sect. 5.1), in the headline's launch configuration."""
    import math
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    n = 32768
    dims = (n, n)
    f, u0 = W.random_smooth_problem_2d_device(n, 2)
    u = torch.empty_like(u0)

    def per_step_ms(p, k):
        u.copy_(u0); p.steps(f, u, 0, k)  # warm-up
        u.copy_(u0); _, m1 = _timed(stream, lambda: p.steps(f, u, 0, k))
        u.copy_(u0); _, m2 = _timed(stream, lambda: p.steps(f, u, 0, 2 * k))
        return (m2 - m1) / k

    out = {"grid": [n, n], "inputs": "f and g from srj_workloads.random_smooth_problem_2d_device (seed 2), "
                                      "generated on the device"}
    t0 = time.perf_counter()
    omega, q = srj.schedules.for_grid(dims, 10)
    out["planner_s"] = time.perf_counter() - t0
    M = int(q.sum())
    kmin, kmax = srj.kappa_range(dims)
    g10 = srj.schedule_check(omega, q, kmin, kmax)
    cycles_bound = math.ceil(10.0 / -g10)
    # the FP64 sweep kernel does not depend on the weights: time it on a one-step plan
    p64 = srj.Plan(dims, 1.0 / (n + 1), [1.0], [1], None, "fp64fma")
    ms64 = per_step_ms(p64, 32)
    out["fp64"] = {"P": 10, "M": M, "omega_1": float(omega[0]), "us_per_step": ms64 * 1e3,
                   "gupdates_per_s": n * n / (ms64 / 1e3) / 1e9, "sweep_kernel": "k_sweep_f64<2,fma>", "steps_timed": 32,
                   "time_to_tol_s_estimate": ms64 / 1e3 * M * cycles_bound,
                   "time_to_tol_kind": "estimate: M steps x %d cycles (1e-10 / max cycle factor %.3g) x measured "
                                       "per-step time" % (cycles_bound, 10 ** g10)}
    del p64
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    try:
        srj.Plan(dims, 1.0 / (n + 1), omega, q, None, "mixed")
        out["mixed_with_optimal_scheme"] = "accepted"
    except srj.SRJError as e:
        out["mixed_with_optimal_scheme"] = "rejected: %s" % str(e).split(": ", 2)[-1]
    out["mixed_check_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    row = srj.schedules.lookup(2, 4096, 10)
    p32 = srj.Plan(dims, 1.0 / (n + 1), row["omega"], row["q"], row["order"], "mixed")
    p32.set_temporal_depth(T)
    p32.set_sweep_variant(variant)
    ms32 = per_step_ms(p32, steps)
    kname = ("k_sweep_f32_tbq<%d,%d>" % (T, 16 if variant == 3 else 8)) if variant in (1, 3) else \
            ("k_sweep_f32_tb<%d,%d>" % (T, 16 if variant in (2, 5) else 8))
    out["mixed"] = {"scheme": "4096^2 grid's P = 10 row (M = %d)" % len(row["order"]), "temporal_depth": T,
                    "sweep_variant": variant, "steps_timed": steps, "us_per_step": ms32 * 1e3,
                    "gupdates_per_s": n * n / (ms32 / 1e3) / 1e9,
                    "roofline": _hbm_roofline(kname, 12 * n * n, ms32 * 1e3 * T, peaks)}
    out["speedup_fp32_vs_fp64_per_step"] = ms64 / ms32
    del p32, f, u0, u
    torch.cuda.empty_cache()
    return {"2d_poisson_32768x32768_P10_throughput": out}


def secondary_workloads(stream, peaks, T, variant):
    """The other configurations: 128^2 FP64, 3-D 512^3, the spherical operator,
    the adjoint, the batch, and the 2^15-per-dimension throughput line."""
    import torch
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    runs = [("config1", lambda: config1_workload(stream, peaks)),
            ("3d", lambda: workload_3d(stream, peaks)),
            ("spherical", lambda: spherical_workload(stream, peaks)),
            ("adjoint", lambda: adjoint_workload(stream, peaks, sm_count, peaks.get("sm_max_mhz", 2070.0))),
            ("batch", lambda: batched_workload(stream, peaks, comparators=True)),
            ("2^15", lambda: large_grid_workload(stream, peaks, T, variant))]
    for name, fn in runs:
        try:
            out.update(fn())
        except Exception as e:  # one failed line must not hide the others
            out[name + "_error"] = "%s: %s" % (type(e).__name__, e)
        torch.cuda.empty_cache()
    return out


def batched_workload(stream, peaks=None, comparators=False, depth=None):
    """One timed solve of the batched workload: 256 problems, n in {64..1024},
    P in 5..10, mixed precision, tol 1e-10 (after one untimed solve).  With
    comparators: the same problems solved one mixed plan at a time (measured),
    and by plain FP64 plans (each problem's FP64 cycle timed, times the cycles
    that problem needed in the batch).  depth: a fixed temporal depth instead
    of the depth tuner's (for profiling runs)."""
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W
    out = {}
    specs = W.batch_specs()
    probs, fs, u0s = [], [], []
    for nn, P, seed in specs:
        row = srj.schedules.lookup(2, nn, P)
        fh, uh = W.random_smooth_problem_2d(nn, seed)
        probs.append(dict(dims=(nn, nn), h=1.0 / (nn + 1), omega=row["omega"], q=row["q"], order=row["order"]))
        fs.append(torch.from_numpy(fh).cuda()); u0s.append(torch.from_numpy(uh).cuda())
    if depth is None:
        tuned_T, tuned_ms = srj.Batch.tune_depth(probs, fs, u0s, 4, 8, stream=stream)
    else:
        tuned_T, tuned_ms = depth, float("nan")
    batch = srj.Batch(probs, temporal_depth=tuned_T)
    us = [x.clone() for x in u0s]
    batch.solve(fs, us, 1e-10, 500)  # warm-up
    us = [x.clone() for x in u0s]
    (stats, dms, rc), ms = _timed(stream, lambda: batch.solve(fs, us, 1e-10, 500))
    info = batch.info()
    T = info["temporal_depth"]
    upd = sum(s_["sweeps"] * nn * nn for s_, (nn, _, _) in zip(stats, specs))
    line = {"time_to_tol_s": ms / 1e3, "gupdates_per_s": upd / (ms / 1e3) / 1e9, "status": rc,
            "max_cycles": max(s_["cycles"] for s_ in stats), "points": sum(nn * nn for nn, _, _ in specs),
            "temporal_depth": T, "depth_tuner": ("srj_batch_tune_depth over T = 4..8 (one cycle of every problem "
                                                 "each): T = %d, %.1f ms per cycle" % (tuned_T, tuned_ms))
                                                if depth is None else "not run: depth fixed at %d" % depth,
            "device_ms": dms,
            "max_final_rel_residual": max(s_["rel_res"] for s_ in stats)}
    if peaks is not None:
        # every launched tile moves its problem's e in, r in, e out once per T steps
        line["roofline"] = _hbm_roofline(
            "k_batch_sweep_grp<%d>" % T, 12.0 * upd / T, dms * 1e3, peaks,
            "achieved over the whole batch solve's device time (one launch = the whole solve; the grouped "
            "sweep is ~92% of it in the ncu launch list)")
        line["roofline"]["algorithmic_bytes_per_launch"] = 12.0 * upd / T
    if comparators:
        one_ms, f64_ms = 0.0, 0.0
        for (nn, P, seed), pr, f, u0, st in zip(specs, probs, fs, u0s, stats):
            p = srj.Plan(pr["dims"], pr["h"], pr["omega"], pr["q"], pr["order"], "mixed")
            p.set_temporal_depth(T)
            u = u0.clone()
            _, m = _timed(stream, lambda: p.solve(f, u, 1e-10, 500))
            one_ms += m
            del p
            p64 = srj.Plan(pr["dims"], pr["h"], pr["omega"], pr["q"], pr["order"], "fp64fma")
            u = u0.clone()
            s64, m64 = _timed(stream, lambda: p64.solve(f, u, 0.0, 1, raise_on_fail=False))
            f64_ms += (m64 - s64["sweep_ms"]) + s64["sweep_ms"] * st["cycles"]
            del p64
        line["one_plan_at_a_time"] = {"time_to_tol_s": one_ms / 1e3, "kind": "measured: each problem's mixed solve "
                                      "(its own plan, same depth), summed"}
        line["fp64_comparator"] = {"time_to_tol_s": f64_ms / 1e3, "kind": "extrapolated: each problem's FP64 cycle "
                                   "timed, times the cycles it needed in the batch, plus its measured set-up; summed"}
        line["speedup_vs_one_plan_at_a_time"] = one_ms / ms
        line["speedup_vs_fp64_time_to_tol"] = f64_ms / ms
    out["batched_256_problems_n64-1024_P5-10_mixed_tol1e-10"] = line
    return out


def oracle_sample(args, sweeps):
    """`sweeps` FP64 oracle sweeps on the full grid; returns (Gupdates/s, seconds)."""
    import numpy as np
    import oracle
    import paper_1511_04292_gb300.schedules as sch
    import srj_workloads as W
    dims = (args.n, args.n)
    f, u = W.random_smooth_problem_2d(args.n, SEED_F)
    row = sch.lookup(2, args.n, args.P)
    seq = oracle.omega_sequence(row["omega"], row["order"])
    oracle.build()
    t0 = time.perf_counter()
    oracle.steps(dims, 1.0 / (args.n + 1), seq, f, u, first=0, count=sweeps)
    dt = time.perf_counter() - t0
    return sweeps * args.n * args.n / dt / 1e9, dt


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    vals = []
    for i in range(args.warmup + args.steps):
        g, dt = oracle_sample(args, args.ref_sweeps)
        if i >= args.warmup:
            vals.append((g, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "Gupdates/s", "cores": 1, "kind": "oracle",
                             "sample": "%d FP64 sweeps of the full %dx%d grid per step" % (args.ref_sweeps, args.n, args.n)},
            "e2e": {"value": value, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_srj(args):
    import numpy as np
    import torch
    import paper_1511_04292_gb300 as srj
    import srj_workloads as W

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    n = args.n
    dims = (n, n)
    pts = n * n
    f_h, u0_h = W.random_smooth_problem_2d(n, SEED_F)
    f = torch.from_numpy(f_h).cuda()
    u0 = torch.from_numpy(u0_h).cuda()
    u = torch.empty_like(u0)
    plan = srj.Plan.from_table(dims, args.P, "mixed")
    if args.T is not None:
        plan.set_temporal_depth(args.T)
        plan.set_sweep_variant(args.variant or 0)
        tuned_T, tuned_us = args.T, None
    else:
        tuned_T, tuned_us = plan.autotune()
    tuned_variant = plan.sweep_variant()
    M = plan.info()["M"]
    launches_per_cycle = -(-M // tuned_T)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    stream = torch.cuda.current_stream()

    def one_solve():
        u.copy_(u0)
        return plan.solve(f, u, TOL, MAX_CYCLES)

    for _ in range(args.warmup):
        st = one_solve()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            stats.append(one_solve())
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.summary()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    sweeps = sum(s["sweeps"] for s in stats)
    sweep_ms = sum(s["sweep_ms"] for s in stats)
    from paper_1511_04292_gb300 import replicas
    value, total_ms, _ = replicas.throughput(total_ms, float(sweeps * pts), device="cuda")
    ms_per_step = total_ms / args.steps

    # dominant kernel: the FP32 sweep; one launch applies T steps to every point
    # and moves e in, r in, e out once: 12 algorithmic bytes per point per launch
    peaks, peak_kind = measured_peaks()
    launches = sum(s["cycles"] for s in stats) * launches_per_cycle
    launch_avg_ms = sweep_ms / launches
    achieved = 12.0 * pts / (launch_avg_ms / 1e3) / 1e9
    if tuned_T == 1:
        kname = "k_sweep_f32<2>"
    elif tuned_variant in (1, 3):
        kname = "k_sweep_f32_tbq<%d,%d>" % (tuned_T, 16 if tuned_variant == 3 else 8)
    else:
        kname = "k_sweep_f32_tb<%d,%d>" % (tuned_T, 16 if tuned_variant == 2 else 8)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": MEASURED_TRAFFIC.get((kname, n)),
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": 12 * pts,
                "avg_launch_us": launch_avg_ms * 1e3, "steps_per_launch": tuned_T,
                "effective_gbs_per_step": 12.0 * pts * sweeps / (sweep_ms / 1e3) / 1e9}

    # end to end through the C ABI with host buffers (srj_solve_host): H2D f, u0; solve; D2H u, all inside
    f_pin = torch.from_numpy(f_h).pin_memory()
    u_pin = torch.from_numpy(u0_h).pin_memory()
    plan.solve_host(f_pin, u_pin, TOL, MAX_CYCLES)  # first call allocates the plan's staging buffers
    e2e_ms = []
    e2e_sweeps = 0
    for i in range(args.steps):
        flush.fill_(float(i))
        u_pin.copy_(torch.from_numpy(u0_h))  # host-side reset of the initial guess, outside the timed region
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = plan.solve_host(f_pin, u_pin, TOL, MAX_CYCLES)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        e2e_sweeps += st["sweeps"]
    e2e_value = world * e2e_sweeps * pts / (sum(e2e_ms) / 1e3) / 1e9

    # plain FP64 SRJ comparator on the same grid and schedule (FP64 steps with fused multiply-adds, the faster
    # of the two FP64 forms)
    p64 = srj.Plan.from_table(dims, args.P, "fp64fma")
    u.copy_(u0)
    torch.cuda.synchronize()
    c64 = args.fp64_cycles if args.fp64_cycles > 0 else MAX_CYCLES
    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st64 = p64.solve(f, u, TOL if args.fp64_cycles == 0 else 0.0, c64, raise_on_fail=False)
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    g64 = st64["sweeps"] * pts / (ms64 / 1e3) / 1e9
    cyc_mixed = stats[-1]["cycles"]
    fp64 = {"gupdates_per_s": g64, "cycles_timed": st64["cycles"], "ms": ms64, "sweep_kernel": "k_sweep_f64<2,fma>",
            "sweep_kernel_gbs": 24.0 * pts / (st64["sweep_ms"] / st64["sweeps"] / 1e3) / 1e9,
            "time_to_tol_s": (ms64 / 1e3 if args.fp64_cycles == 0 else ms64 / 1e3 / st64["cycles"] * cyc_mixed),
            "time_to_tol_kind": "measured" if args.fp64_cycles == 0 else
            "per-cycle time x the %d cycles the mixed solve needed (same cycle map in exact arithmetic)" % cyc_mixed}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, dt = oracle_sample(args, args.cpu_sweeps)
        sweeps_solve = stats[-1]["sweeps"]
        cpu = {"value": g, "unit": "Gupdates/s", "cores": 1, "kind": "oracle",
               "sample": "%d FP64 oracle sweeps of the full %dx%d grid (%.1f s)" % (args.cpu_sweeps, n, n, dt),
               "host_cores_total": os.cpu_count(),
               "time_to_tol_s_extrapolated": sweeps_solve * pts / (g * 1e9),
               "time_to_tol_kind": "extrapolated: the oracle's measured per-sweep time x the %d sweeps the GPU "
                                   "solve needed (FP64 SRJ needs the same cycles in exact arithmetic)" % sweeps_solve}

    secondary = None
    if rank == 0 and not args.no_secondary:
        del p64
        torch.cuda.empty_cache()
        secondary = secondary_workloads(stream, peaks, tuned_T, tuned_variant)

    launches_per_step = 2 + stats[-1]["cycles"] * (launches_per_cycle + 2)
    line = {"metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "time_to_tol_s": ms_per_step / 1e3, "temporal_depth": tuned_T, "sweep_variant": tuned_variant, "autotune_us_per_step": tuned_us, "cycles": stats[-1]["cycles"], "sweeps_per_solve": stats[-1]["sweeps"],
            "final_rel_residual": stats[-1]["rel_res"],
            "fp64_comparator": fp64, "speedup_vs_fp64_time_to_tol": fp64["time_to_tol_s"] / (ms_per_step / 1e3),
            "roofline": roofline, "clocks": clocks, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "Gupdates/s", "h2d_bytes_per_step": 2 * f_h.nbytes,
                    "d2h_bytes_per_step": u0_h.nbytes, "ms_per_step": sum(e2e_ms) / len(e2e_ms),
                    "call": "srj_solve_host (pinned host f, u)"},
            "gpu_launches": launches_per_step * args.steps, "secondary_workloads": secondary}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.kernel_case:
        return run_kernel_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_srj(args)


if __name__ == "__main__":
    sys.exit(main())
