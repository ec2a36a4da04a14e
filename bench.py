"""Benchmark of the MRI fast-partition solve on GB300.

Workload (synthetic, seeded): the 32^3 periodic box -- 40 species / 170
reactions (12 third-body, 8 Troe falloff), temperature from 8 Gaussian hot
spots (300..2500 K), Dirichlet mass fractions, 4th-order central
advection-diffusion as the slow partition, explicit MRI3 (Knoth-Wolke, MIS form)
with SDIRK3 fast substeps, H = 5e-8 s, h = H/10, Newton tolerance 1e-10.
One bench step = one MRI slow step over the whole box (three f^S evaluations,
three stage forcings, three fast stages) through the C ABI.

Metric: fast-chemistry cell-steps per second, a cell-step being one SDIRK
substep of one cell (all its stages and Newton iterations), counted from the
kernels' own per-cell counters.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch one process per GPU with torch.distributed.run; every rank
integrates its own replica of the box (weak scaling, no data-path collective).
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

METRIC = "fast-chem cell-steps/s per MRI slow step, plain FP64 vs tuned, at rel err ≤1e-6"
UNIT = "cell-steps/s"
WORKLOAD = "box32"
# FP64 roofline: the FMA pipe issues 2 DFMA per clock per SM on GB300 (measured, see the
# alu_fp64 profile), 152 SMs, 2 flops per FMA; at the maximum SM clock of 2070 MHz this is
# the figure below.  The bench also measures the rate live (mri_probe_fp64_fma) and uses
# that measurement as the peak.
FP64_DFMA_PER_CLK_SM = 2.0
N_SM = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS_NOMINAL = FP64_DFMA_PER_CLK_SM * 2 * N_SM * SM_MAX_MHZ * 1e6 / 1e12
# nominal cost of one exp or log in the algorithmic flop count
FLOPS_PER_TRANSCENDENTAL = 20.0


# ----------------------------------------------------------------------------- flop model

def flop_model(mech):
    """Algorithmic FP64 flops of the pieces of one fast substep for a mechanism:
    (f^F evaluation, Jacobian assembly + Newton matrix, LU factorisation, one
    Newton solve + update).  Counted from the mechanism's structure; exp/log at
    FLOPS_PER_TRANSCENDENTAL each."""
    E = FLOPS_PER_TRANSCENDENTAL
    Ns, R = mech.n_species, mech.n_reactions
    n = Ns + 1
    nreac = (mech.reac >= 0).sum(1)
    nprod = (mech.prod >= 0).sum(1)
    ntroe = int((mech.rtype == 2).sum())
    ntb = int((mech.rtype != 0).sum())
    # net stoichiometric incidences (species appearing with nu != 0)
    inc = 0
    col = 0
    for r in range(R):
        net = {}
        for i in mech.reac[r]:
            if i >= 0:
                net[i] = net.get(i, 0) - 1
        for i in mech.prod[r]:
            if i >= 0:
                net[i] = net.get(i, 0) + 1
        inc += sum(1 for v in net.values() if v != 0)
        col += len(net)
    eff_dev = int(sum((row != 1.0).sum() for row in mech.eff)) if mech.eff.size else 0
    rates = (2 * Ns + 6                       # S, concentrations
             + Ns * 30                        # cp, h, s, g polynomials
             + E                              # ln T
             + R * (8 + 4 + 2 * E)            # sum nu g, ln k, ln Kc, k_f, k_r
             + int((nreac + nprod).sum())     # rate products
             + 3 * R                          # q
             + 2 * eff_dev + ntb              # [M]
             + ntroe * (7 * E + 40)           # falloff
             + 2 * inc                        # production rates
             + 4 * Ns + 10)                   # f
    jac = (rates + R * 12 + ntroe * 40         # rate derivatives
           + col * 8 + 2 * inc * 3             # dq/dC and nu scatter
           + 2 * ntb * Ns * 3                  # third-body columns
           + 4 * Ns * Ns + 10 * Ns             # DC, column sums, chain rule
           + 2 * n * n)                        # M = I - hg J
    lu = (2.0 / 3.0) * n ** 3 + n
    solve = 2 * n * n + 8 * n
    return dict(rates=rates, jac=jac, lu=lu, solve=solve, n=n)


def algorithmic_flops(fm, substeps, newton, njac):
    """Flops of a batch of substeps from the per-cell counters: every Newton
    iteration costs one f^F evaluation and one solve; every Jacobian evaluation
    costs an assembly and a factorisation."""
    return newton * (fm["rates"] + fm["solve"]) + njac * (fm["jac"] + fm["lu"])


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def gpu_arm(args, rank, world):
    import torch

    import mechgen
    import paper_2211_03293_gb300 as mri

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = mechgen.workload(WORKLOAD, seed=0, cells_per_side=args.cells_per_side)
    g = w.grid
    ncell = w.y0.shape[0]
    n = w.mech.n
    mech = mri.mri_mech_load(w.mech.to_blob())
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    c, G = mri.mri_method_coupling(mri.MRI_KW3)
    stream = torch.cuda.Stream(device=dev)
    y = torch.tensor(w.y0, device=dev)
    p = torch.tensor(w.p, device=dev)
    fS = torch.empty((3, ncell, n), dtype=torch.float64, device=dev)
    phi = torch.empty((ncell, 1, n), dtype=torch.float64, device=dev)
    stats = torch.zeros((ncell, 4), dtype=torch.int32, device=dev)
    status = torch.zeros(ncell, dtype=torch.int32, device=dev)
    nfail = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)    # 256 MB > 129 MB L2
    probe = torch.empty(N_SM * 8 * 256 * 4, dtype=torch.float64, device=dev)
    fp64_peak_tflops = 2.0 * mri.mri_probe_fp64_fma(probe, iters=4096) / 1e12
    H, h = w.H, w.h
    base_opts = mri.mri_fast_opts_default(method=w.method, newton_rtol=w.newton_rtol, jac_policy=args.jac,
                                          precision=args.prec)
    ramp_opts = mri.mri_fast_opts_default(method=w.method, newton_rtol=w.newton_rtol, ramp=w.ramp,
                                          jac_policy=args.jac, precision=args.prec)

    def mri_step_timed(first, ev_stage):
        """One MRI slow step through the ABI; CUDA events around each fast stage."""
        for i in range(1, 4):
            mri.mri_slow_rhs(y, fS[i - 1], grid, stream=stream)
            mri.mri_stage_forcing(fS, i, G[i], phi, stream=stream)
            o = ramp_opts if (first and i == 1) else base_opts
            if ev_stage is not None:
                ev_stage[i - 1][0].record(stream)
            mri.mri_stage_fast(y, p, phi, 0.0, (c[i] - c[i - 1]) * H, h, mech, o, cell_status=status,
                               cell_stats=stats, n_failed=nfail, stream=stream)
            if ev_stage is not None:
                ev_stage[i - 1][1].record(stream)

    with torch.cuda.stream(stream):
        for s in range(args.warmup):
            mri_step_timed(s == 0, None)
        stream.synchronize()
        warm_fail = int(nfail.item())
        stats.zero_()
        y_start = y.clone()          # the e2e leg replays the timed steps from this state
        kernel_launches_per_step = 9
        step_events = []
        stage_events = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = str(dev.index)
        sampler = ClockSampler(gpu_id)
        sampler.start()
        for s in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            e0.record(stream)
            mri_step_timed(args.warmup == 0 and s == 0, ev)
            e1.record(stream)
            step_events.append((e0, e1))
            stage_events.append(ev)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if world > 1:
            torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in step_events]
    stage_ms = [[a.elapsed_time(b) for a, b in ev] for ev in stage_events]
    st = stats.cpu().numpy().astype(np.int64)
    substeps = int(st[:, 0].sum())
    newton = int(st[:, 1].sum())
    njac = int(st[:, 2].sum())
    failed = int(nfail.item()) - warm_fail
    total_ms = float(sum(step_ms))

    # end to end through the public C-ABI call with host buffers: the same K steps from
    # the same state, each step copying the state in from pinned host memory and the
    # result back
    y_host = torch.empty((ncell, n), dtype=torch.float64, pin_memory=True)
    y_host.copy_(y_start.cpu())
    p_host = torch.empty(ncell, dtype=torch.float64, pin_memory=True)
    p_host.copy_(p.cpu())
    ws = torch.empty(mri.mri_step_workspace_size(grid, n) // 8, dtype=torch.float64, device=dev)
    e2e_stats = torch.zeros((ncell, 4), dtype=torch.int32, device=dev)
    e2e_ms = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y.copy_(y_host, non_blocking=True)
            p.copy_(p_host, non_blocking=True)
            mri.mri_step(y, p, grid, s * H, H, h, mech, base_opts, ws, cell_stats=e2e_stats, stream=stream)
            y_host.copy_(y, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_sub = int(e2e_stats[:, 0].sum().item())

    fm = flop_model(w.mech)
    flops_all = algorithmic_flops(fm, substeps, newton, njac)
    stage_total_ms = float(np.sum(stage_ms))
    launches = 3 * args.steps
    res = dict(total_ms=total_ms, substeps=substeps, newton=newton, njac=njac, failed=failed, clocks=clocks,
               step_ms=step_ms, stage_total_ms=stage_total_ms, stage_launches=launches, flops=flops_all,
               e2e_ms=float(sum(e2e_ms)), e2e_substeps=e2e_sub, ncell=ncell, n=n,
               launches=kernel_launches_per_step * args.steps, h2d=(ncell * n + ncell) * 8, d2h=ncell * n * 8,
               workload=w, fp64_peak_tflops=fp64_peak_tflops)
    return res


def cpu_baseline_sample(ncells_sample, seed=0, nthreads=None, repeats=1):
    """The oracle on a bounded sample of the same workload: the three fast stages
    of one MRI step (forcing f^S(y0) from the oracle's slow stencil) on randomly
    sampled cells, after an untimed start-up stage."""
    import mechgen
    import oracle

    w = mechgen.workload(WORKLOAD, seed=0)
    m = oracle.Mech(w.mech)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.y0.shape[0], ncells_sample, replace=False))
    fS = oracle.slow_rhs(w.y0, w.grid)[idx][:, None, :]
    y = w.y0[idx]
    p = w.p[idx]
    nthreads = nthreads or os.cpu_count() or 1
    o0 = oracle.opts(method=w.method, rtol=w.newton_rtol, ramp=w.ramp)
    o = oracle.opts(method=w.method, rtol=w.newton_rtol)
    y, st, _ = m.stage_fast(y, p, fS, w.H / 3, w.h, o0, nthreads=nthreads)
    cs, tt = 0, 0.0
    for _ in range(repeats):
        for dc in (1 / 3, 5 / 12, 1 / 4):
            t0 = time.perf_counter()
            y, st, stats = m.stage_fast(y, p, fS, dc * w.H, w.h, o, nthreads=nthreads)
            tt += time.perf_counter() - t0
            cs += int(stats[:, 0].sum())
    return cs / tt, nthreads, cs, tt


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4096, help="cells of the oracle's CPU baseline sample")
    ap.add_argument("--cells-per-side", type=int, default=None,
                    help="shrink the box (profiling captures only; the bench line is for 32^3)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling captures)")
    ap.add_argument("--jac", type=int, default=1, help="Newton matrix policy: 0 per substep, 1 lazy")
    ap.add_argument("--prec", type=int, default=0, help="0 plain FP64, 1 FP32 Jacobian/LU with FP64 residual")
    args = ap.parse_args()
    rank, world = dist_init(args)

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build.build()
        vals = []
        t_all = 0.0
        cs_all = 0
        cores = os.cpu_count() or 1
        for s in range(args.warmup + args.steps):
            v, cores, cs, tt = cpu_baseline_sample(256, seed=100 + s)
            if s >= args.warmup:
                vals.append(v)
                t_all += tt
                cs_all += cs
        value = cs_all / t_all
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": "box32 (32^3 cells, 40 species / 170 reactions, MRI3 + SDIRK3, "
                                       "H = 5e-8 s, h = H/10)", "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": "per step: the three fast stages of one MRI step on 256 sampled cells "
                                           "(forcing from the oracle's slow stencil) after an untimed start-up "
                                           "stage"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    res = gpu_arm(args, rank, world)
    # max time over ranks, sum of work
    t = torch.tensor([res["total_ms"], res["e2e_ms"]], dtype=torch.float64, device="cuda")
    work = torch.tensor([res["substeps"], res["e2e_substeps"]], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(work, op=torch.distributed.ReduceOp.SUM)
    t = t.cpu().numpy()
    work = work.cpu().numpy()
    if rank != 0:
        return
    value = work[0] / (t[0] * 1e-3)
    e2e_value = work[1] / (t[1] * 1e-3)
    # roofline of the dominant kernel (the fast stage): algorithmic flops per launch
    # over its average event-timed duration
    flops_per_launch = res["flops"] / res["stage_launches"]
    avg_launch_s = res["stage_total_ms"] * 1e-3 / res["stage_launches"]
    achieved = flops_per_launch / avg_launch_s / 1e12
    peak = res["fp64_peak_tflops"]
    if args.no_cpu:
        cpu_v, cores, cs, tt = None, 0, 0, 0.0
    else:
        cpu_v, cores, cs, tt = cpu_baseline_sample(args.cpu_sample)
    w = res["workload"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "box32: 32^3 periodic box, 40 species / 170 reactions (12 third-body, 8 Troe), "
                               "MRI3 (Knoth-Wolke MIS) + SDIRK3 fast, H = 5e-8 s, h = H/10, Newton rtol 1e-10, "
                               "4th-order slow stencil; one step = one MRI slow step",
                   "cells": res["ncell"], "unknowns_per_cell": res["n"],
                   "form": ["plain FP64", "mixed: FP32 Jacobian/LU, FP64 rates/residual"][args.prec],
                   "jac_policy": ["per-substep", "lazy"][args.jac],
                   "reduced_for_profiling": args.cells_per_side is not None,
                   "l2": "256 MB buffer written between timed steps",
                   "newton_per_substep": res["newton"] / max(res["substeps"], 1),
                   "jac_per_substep": res["njac"] / max(res["substeps"], 1),
                   "failed_cells": res["failed"]},
        "clocks": res["clocks"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "stage_fast_kernel",
                     "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_launch_s * 1e3,
                     "peak_basis": "FP64 FMA pipe rate measured in this run (mri_probe_fp64_fma; the pipe "
                                   "issues 2 DFMA/clk/SM, %.4f TFLOP/s at 2070 MHz); MEASURED_PEAKS.json has no "
                                   "FP64 entry" % FP64_PEAK_TFLOPS_NOMINAL},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"the three fast stages of one MRI step on {args.cpu_sample} sampled cells "
                                   f"({cs} cell-steps, {tt:.1f} s), forcing from the oracle's slow stencil, after "
                                   f"an untimed start-up stage"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": res["launches"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
