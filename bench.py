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
kernels' own per-cell counters.  Three forms are timed: the plain FP64 path,
the mixed-precision path (FP32 Newton matrix / LU, FP64 rates and residual) and
the learned start on the mixed path (a bf16 network trained on the first steps
predicts Newton starts; its inference is inside the timed steps).  Each form
uses the persistent kernel's autotuned launch shape and keeps Newton matrices
across calls, and is gated against the CPU oracle (sampled cells of a full-size
stage, relative error <= 1e-6, per-field maxima and RMS reported); the headline
is the fastest form that passes.

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
GATE_TOL = 1e-6
# FP64 roofline: the FMA pipe issues 2 DFMA per clock per SM on GB300 (measured), 152 SMs,
# 2 flops per FMA; at the maximum SM clock of 2070 MHz this is the figure below.  The bench
# measures the rate live (mri_probe_fp64_fma) and uses that measurement as the peak.
FP64_DFMA_PER_CLK_SM = 2.0
N_SM = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS_NOMINAL = FP64_DFMA_PER_CLK_SM * 2 * N_SM * SM_MAX_MHZ * 1e6 / 1e12
# nominal cost of one exp or log in the algorithmic flop count
FLOPS_PER_TRANSCENDENTAL = 20.0
# DRAM bytes (read + write) per cell and fast-stage launch of stage_fast_kernel with the
# Newton-matrix cache in use, from the ncu captures summarised in
# profiles/stage_fast_fp64_box16.md and profiles/stage_fast_mixed_box16.md (4096-cell
# launches; traffic grows with the cells processed, so a launch over `cells` moves
# cells times this).  Keep in step with the kernel: a changed kernel needs a new
# capture before these figures are reported again.
STAGE_DRAM_BYTES_PER_CELL = {0: (61920512 + 2869504) / 4096, 1: (33669888 + 3328) / 4096}
FORMS = {0: "plain FP64", 1: "mixed: FP32 Newton matrix and LU, FP64 rates, residual and update",
         2: "learned: mixed form with Newton started from a bf16 MLP's prediction where the predictor has none"}


# ----------------------------------------------------------------------------- flop model

def flop_model(mech):
    """Algorithmic flops of the pieces of one fast substep for a mechanism:
    f^F evaluation (rates), the FP64 extras of a Jacobian evaluation (rate
    derivatives), the Jacobian assembly proper, LU, and one Newton solve; plus the
    FP64 vector work of a Newton iteration (residual, update, norm).  Counted from
    the mechanism's structure; exp/log at FLOPS_PER_TRANSCENDENTAL each."""
    E = FLOPS_PER_TRANSCENDENTAL
    Ns, R = mech.n_species, mech.n_reactions
    n = Ns + 1
    nreac = (mech.reac >= 0).sum(1)
    nprod = (mech.prod >= 0).sum(1)
    ntroe = int((mech.rtype == 2).sum())
    ntb = int((mech.rtype != 0).sum())
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
    jac_fp64 = R * 12 + ntroe * 40 + 2 * inc   # rate derivatives and sum nu dq/dT
    jac_asm = (col * 8 + 2 * inc * 3           # dq/dC and nu scatter
               + 2 * ntb * Ns * 3              # third-body columns
               + 4 * Ns * Ns + 10 * Ns         # DC, column sums, chain rule
               + 2 * n * n)                    # M = I - hg J
    lu = (2.0 / 3.0) * n ** 3 + n
    solve = 2 * n * n
    vec = 8 * n                                # residual, update, WRMS norm
    return dict(rates=rates, jac_fp64=jac_fp64, jac_asm=jac_asm, lu=lu, solve=solve, vec=vec, n=n)


def algorithmic_flops(fm, newton, njac, prec):
    """(FP64 flops, FP32 flops) of a batch of substeps from the per-cell counters:
    every Newton iteration costs an f^F evaluation, a solve and the vector work;
    every Jacobian evaluation costs an f^F evaluation with derivatives, the
    assembly and a factorisation.  The mixed form runs assembly, LU and solves in
    FP32."""
    fp64 = newton * (fm["rates"] + fm["vec"]) + njac * (fm["rates"] + fm["jac_fp64"])
    mat = newton * fm["solve"] + njac * (fm["jac_asm"] + fm["lu"])
    return (fp64 + mat, 0.0) if prec == 0 else (fp64, mat)


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

class Bench:
    def __init__(self, args, world):
        import torch

        import mechgen
        import paper_2211_03293_gb300 as mri

        self.mri, self.torch, self.args, self.world = mri, torch, args, world
        self.dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(self.dev)
        self.w = w = mechgen.workload(WORKLOAD, seed=0, cells_per_side=args.cells_per_side)
        g = w.grid
        self.ncell = w.y0.shape[0]
        self.n = w.mech.n
        self.mech = mri.mri_mech_load(w.mech.to_blob())
        self.grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
        self.c, self.G = mri.mri_method_coupling(mri.MRI_KW3)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.shape = {}
        self.cache = {}
        dev = self.dev
        self.p = torch.tensor(w.p, device=dev)
        self.fS = torch.empty((3, self.ncell, self.n), dtype=torch.float64, device=dev)
        self.phi = torch.empty((self.ncell, 1, self.n), dtype=torch.float64, device=dev)
        self.stats = torch.zeros((self.ncell, 4), dtype=torch.int32, device=dev)
        self.status = torch.zeros(self.ncell, dtype=torch.int32, device=dev)
        self.nfail = torch.zeros(1, dtype=torch.int32, device=dev)
        self.nfallback = torch.zeros(1, dtype=torch.int32, device=dev)
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)    # 256 MB > 129 MB L2
        probe = torch.empty(N_SM * 8 * 256 * 4, dtype=torch.float64, device=dev)
        self.fp64_peak_tflops = 2.0 * mri.mri_probe_fp64_fma(probe, iters=4096) / 1e12
        try:
            self.gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            self.gpu_id = str(dev.index)

    def newton_safety(self, prec):
        """The plain FP64 form keeps the library's default acceptance of modified-Newton
        iterates; the tuned forms (mixed and learned) use the bench's setting."""
        return 3e-4 if prec == 0 else self.args.tuned_newton_safety

    def opts(self, prec, ramp=0):
        w = self.w
        wpb, bps = self.shape.get(prec, (0, 0))
        o = self.mri.mri_fast_opts_default(method=w.method, newton_rtol=w.newton_rtol, ramp=ramp,
                                           jac_policy=self.args.jac, precision=prec, warps_per_block=wpb,
                                           blocks_per_sm=bps, newton_safety=self.newton_safety(prec))
        cache = self.cache.get(prec)
        return o if cache is None else self.mri.with_matrix_cache(o, cache)

    def autotune(self, y, prec):
        """Pick the launch shape of the fast stage by timing the candidates on the
        first stage of the next step (copies of the state and of its forcing)."""
        from paper_2211_03293_gb300.autotune import autotune_stage
        mri, c, G, w = self.mri, self.c, self.G, self.w
        with self.torch.cuda.stream(self.stream):
            mri.mri_slow_rhs(y, self.fS[0], self.grid, stream=self.stream)
            mri.mri_stage_forcing(self.fS, 1, G[1], self.phi, stream=self.stream)
            best, table = autotune_stage(self.mech, y, self.p, self.phi, (c[1] - c[0]) * w.H, w.h, self.opts(prec),
                                         repeats=2, stream=self.stream)
        self.shape[prec] = (best.warps_per_block, best.blocks_per_sm)
        wpb, blocks, smem = mri.mri_stage_fast_shape(self.mech, best, self.ncell, 1)
        return {"warps_per_block": wpb, "blocks": blocks, "blocks_per_sm": max(best.blocks_per_sm, 1),
                "smem_bytes": smem, "autotuned": [[a, b_, round(ms, 3)] for a, b_, ms in table]}

    def graph_steps(self, y, prec):
        """The same MRI step recorded once in a CUDA graph and replayed args.steps times
        (L2 flushed between replays); returns (ms per step, substeps run)."""
        torch, args = self.torch, self.args
        graph = torch.cuda.CUDAGraph()
        self.stream.synchronize()
        with torch.cuda.graph(graph, stream=self.stream):
            self.step(y, prec, False, None)
        self.stats.zero_()
        torch.cuda.synchronize()
        evs = []
        with torch.cuda.stream(self.stream):
            for _ in range(args.steps):
                self.flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                graph.replay()
                e1.record(self.stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        sub = int(self.stats[:, 0].sum().item())
        del graph
        return ms, sub

    def step(self, y, prec, first, ev_stage, model=None):
        """One MRI slow step through the ABI; CUDA events around each fast stage.
        With a learned model every stage first evaluates the network (features,
        forward pass, guess) and starts Newton from its guess where the analytic
        predictor has no derivative yet."""
        mri, c, G, w = self.mri, self.c, self.G, self.w
        for i in range(1, 4):
            mri.mri_slow_rhs(y, self.fS[i - 1], self.grid, stream=self.stream)
            mri.mri_stage_forcing(self.fS, i, G[i], self.phi, stream=self.stream)
            o = self.opts(prec, w.ramp if (first and i == 1) else 0)
            Hs = (c[i] - c[i - 1]) * w.H
            if model is not None:
                guess = model.guess(y, self.p, self.phi, Hs, w.h, stream=self.stream)
            if ev_stage is not None:
                ev_stage[i - 1][0].record(self.stream)
            if model is None:
                mri.mri_stage_fast(y, self.p, self.phi, 0.0, Hs, w.h, self.mech, o, cell_status=self.status,
                                   cell_stats=self.stats, n_failed=self.nfail, stream=self.stream)
            else:
                mri.mri_stage_fast_guided(y, self.p, self.phi, 0.0, Hs, w.h, self.mech, o,
                                          start=mri.MRI_START_GUESS_FIRST, guess=guess, cell_status=self.status,
                                          cell_stats=self.stats, n_failed=self.nfail, n_fallback=self.nfallback,
                                          stream=self.stream)
            if ev_stage is not None:
                ev_stage[i - 1][1].record(self.stream)

    def adaptive_steps(self, y_start, prec, tol=1e-6):
        """The same K steps from the same state with adaptive substeps (controller
        tolerance tol): device time per MRI step and accepted substeps per cell and
        stage, beside the fixed scheme's."""
        torch, mri, args, w, c, G = self.torch, self.mri, self.args, self.w, self.c, self.G
        y = y_start.clone()
        st = torch.zeros((self.ncell, 4), dtype=torch.int32, device=self.dev)
        evs = []
        with torch.cuda.stream(self.stream):
            for s in range(args.steps):
                self.flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                for i in range(1, 4):
                    mri.mri_slow_rhs(y, self.fS[i - 1], self.grid, stream=self.stream)
                    mri.mri_stage_forcing(self.fS, i, G[i], self.phi, stream=self.stream)
                    o = self.opts(prec)
                    o.adaptive, o.ctrl_rtol, o.ctrl_atol_Y, o.ctrl_atol_T = 1, tol, tol * 1e-6, tol
                    mri.mri_stage_fast(y, self.p, self.phi, 0.0, (c[i] - c[i - 1]) * w.H, w.h, self.mech, o,
                                       cell_stats=st, stream=self.stream)
                e1.record(self.stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b_) for a, b_ in evs) / args.steps
        acc = st[:, 0].sum().item() / (3 * args.steps * self.ncell)
        return {"ctrl_rtol": tol, "ms_per_step": ms, "accepted_substeps_per_cell_stage": acc,
                "fixed_substeps_per_cell_stage": 12 / 3,
                "note": "controller tolerance 1e-6 (global stage error about 1e-6 on relaxed states, "
                        "against about 3e-4 for the fixed h = H/10 in the oracle's comparison with "
                        "256x finer steps)"}

    def train_learned(self, prec):
        """The learned form's network, trained by the library's kernels on the
        substep-end states the plain solver produces over the first MRI steps of the
        workload (the start-up step excluded).  Returns (model, training report)."""
        from paper_2211_03293_gb300.learned import LearnedStart, stage_substep_states
        torch, mri, c, G, w, args = self.torch, self.mri, self.c, self.G, self.w, self.args
        t0 = time.time()
        model = LearnedStart(self.n, g_max=5, batch=4096, infer_batch=self.ncell)
        y = torch.tensor(w.y0, device=self.dev)
        with torch.cuda.stream(self.stream):
            for s in range(1 + args.learn_steps):
                for i in range(1, 4):
                    mri.mri_slow_rhs(y, self.fS[i - 1], self.grid, stream=self.stream)
                    mri.mri_stage_forcing(self.fS, i, G[i], self.phi, stream=self.stream)
                    Hs = (c[i] - c[i - 1]) * w.H
                    o = self.opts(prec, w.ramp if (s == 0 and i == 1) else 0)
                    y_in = y.clone()
                    seq, _ = stage_substep_states(y, self.p, self.phi, Hs, w.h, self.mech, o, stream=self.stream)
                    if s > 0:
                        model.add(y_in, self.p, self.phi.clone(), Hs, seq)
            torch.cuda.synchronize()
            t_data = time.time() - t0
            hist = model.fit(epochs=args.learn_epochs, lr=2e-3, stream=self.stream)
        torch.cuda.synchronize()
        rep = {"examples": int(sum(r[0].shape[0] for r in model.records)), "epochs": args.learn_epochs,
               "loss_first": hist[0], "loss_last": hist[-1], "data_s": round(t_data, 2),
               "train_s": round(time.time() - t0 - t_data, 2), "network": model.dims,
               "start": "MRI_START_GUESS_FIRST (network where the analytic predictor has no derivative yet)"}
        return model, rep

    def gate(self, prec, model=None):
        """Relative error of the first fast stage of the full-size workload (forcing
        f^S(y0) from the oracle) on 32 sampled cells against the CPU oracle, with the
        maximum and RMS per field (mass fractions above 1e-10, and T)."""
        import oracle
        torch, mri, w = self.torch, self.mri, self.w
        fS = oracle.slow_rhs(w.y0, w.grid)
        y = torch.tensor(w.y0, device=self.dev)
        ph = torch.tensor(fS[:, None, :].copy(), device=self.dev)
        with torch.cuda.stream(self.stream):
            if model is None:
                mri.mri_stage_fast(y, self.p, ph, 0.0, w.H / 3, w.h, self.mech, self.opts(prec, w.ramp),
                                   stream=self.stream)
            else:
                guess = model.guess(y, self.p, ph, w.H / 3, w.h, stream=self.stream)
                mri.mri_stage_fast_guided(y, self.p, ph, 0.0, w.H / 3, w.h, self.mech, self.opts(prec, w.ramp),
                                          start=mri.MRI_START_GUESS_FIRST, guess=guess, stream=self.stream)
        self.stream.synchronize()
        rng = np.random.default_rng(11)
        idx = np.sort(rng.choice(self.ncell, min(32, self.ncell), replace=False))
        ref, _, _ = oracle.Mech(w.mech).stage_fast(w.y0[idx], w.p[idx], fS[idx][:, None, :], w.H / 3, w.h,
                                                    oracle.opts(method=w.method, rtol=w.newton_rtol, ramp=w.ramp))
        got = y.cpu().numpy()[idx]
        scale = np.abs(ref)
        scale[:, :-1] = np.maximum(scale[:, :-1], 1e-10)
        rel = np.abs(got - ref) / scale
        err = float(np.max(rel))
        big = ref[:, :-1] > 1e-10
        ry, rt = rel[:, :-1][big], rel[:, -1]
        fields = {"Y_max": float(ry.max()), "Y_rms": float(np.sqrt(np.mean(ry ** 2))), "T_max": float(rt.max()),
                  "T_rms": float(np.sqrt(np.mean(rt ** 2)))}
        return {"cells": int(len(idx)), "max_rel_err": err, "tolerance": GATE_TOL, "passed": err <= GATE_TOL,
                "per_field": fields}

    def run_form(self, form):
        """Time one form: 0 plain FP64, 1 mixed precision, 2 learned start on the mixed
        form (network inference inside the timed steps)."""
        torch, mri, args, w = self.torch, self.mri, self.args, self.w
        prec = 1 if form == 2 else form
        model, learn = self.train_learned(prec) if form == 2 else (None, None)
        if args.matrix_cache and args.jac == 1:
            self.cache[prec] = torch.zeros(mri.mri_matrix_cache_size(self.mech, self.ncell, prec),
                                           dtype=torch.uint8, device=self.dev)
        y = torch.tensor(w.y0, device=self.dev)
        with torch.cuda.stream(self.stream):
            for s in range(args.warmup):
                self.step(y, prec, s == 0, None, model)
            self.stream.synchronize()
            launch = self.autotune(y, prec) if (args.autotune and form != 2) else None
            if form == 2 and args.autotune and prec in self.shape:
                launch = {"warps_per_block": self.shape[prec][0], "blocks_per_sm": max(self.shape[prec][1], 1),
                          "autotuned": "shape of the mixed form"}
            if prec in self.cache:
                self.cache[prec].zero_()      # the autotuner's trial runs leave no matrices behind
                for s in range(1):            # one more untimed step refills the cache
                    self.step(y, prec, False, None, model)
            self.stream.synchronize()
            warm_fail = int(self.nfail.item())
            self.stats.zero_()
            self.nfallback.zero_()
            y_start = y.clone()          # the e2e leg replays the timed steps from this state
            step_events, stage_events = [], []
            if self.world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            sampler = ClockSampler(self.gpu_id)
            sampler.start()
            for s in range(args.steps):
                self.flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(3)]
                e0.record(self.stream)
                self.step(y, prec, args.warmup == 0 and s == 0, ev, model)
                e1.record(self.stream)
                step_events.append((e0, e1))
                stage_events.append(ev)
            torch.cuda.synchronize()
            clocks = sampler.stop()
            if self.world > 1:
                torch.distributed.barrier()
        step_ms = [a.elapsed_time(b) for a, b in step_events]
        stage_ms = [[a.elapsed_time(b) for a, b in ev] for ev in stage_events]
        st = self.stats.cpu().numpy().astype(np.int64)
        substeps, newton, njac = int(st[:, 0].sum()), int(st[:, 1].sum()), int(st[:, 2].sum())
        failed = int(self.nfail.item()) - warm_fail
        fallbacks = int(self.nfallback.item())
        graph_ms, graph_sub = (self.graph_steps(y_start.clone(), prec) if (args.graph and form != 2)
                               else (None, None))

        # end to end through the public C-ABI call with host buffers: the same K steps
        # from the same state, each step copying the state in from pinned host memory
        # and the result back
        n, ncell = self.n, self.ncell
        y_host = torch.empty((ncell, n), dtype=torch.float64, pin_memory=True)
        y_host.copy_(y_start.cpu())
        p_host = torch.empty(ncell, dtype=torch.float64, pin_memory=True)
        p_host.copy_(self.p.cpu())
        ws = torch.empty(mri.mri_step_workspace_size(self.grid, n) // 8, dtype=torch.float64, device=self.dev)
        e2e_stats = torch.zeros((ncell, 4), dtype=torch.int32, device=self.dev)
        e2e_ms = []
        with torch.cuda.stream(self.stream):
            for s in range(args.steps):
                self.flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                y.copy_(y_host, non_blocking=True)
                self.p.copy_(p_host, non_blocking=True)
                if model is None:
                    mri.mri_step(y, self.p, self.grid, s * w.H, w.H, w.h, self.mech, self.opts(prec), ws,
                                 cell_stats=e2e_stats, stream=self.stream)
                else:
                    saved, self.stats = self.stats, e2e_stats
                    self.step(y, prec, False, None, model)
                    self.stats = saved
                y_host.copy_(y, non_blocking=True)
                e1.record(self.stream)
                e1.synchronize()
                e2e_ms.append(e0.elapsed_time(e1))
        e2e_sub = int(e2e_stats[:, 0].sum().item())
        adaptive = self.adaptive_steps(y_start, prec) if (args.adaptive and model is None) else None
        fm = flop_model(w.mech)
        f64, f32 = algorithmic_flops(fm, newton, njac, prec)
        # kernels per step: 3 x (stencil, forcing, stage) [+ 3 x (features, input conversion,
        # 4 GEMMs, guess) for the learned form]
        per_step = 9 + (18 if model is not None else 0)
        return dict(prec=prec, form=form, total_ms=float(sum(step_ms)), substeps=substeps, newton=newton,
                    njac=njac, failed=failed, clocks=clocks, stage_total_ms=float(np.sum(stage_ms)),
                    stage_launches=3 * args.steps, flops64=f64, flops32=f32, e2e_ms=float(sum(e2e_ms)),
                    e2e_substeps=e2e_sub, launches=per_step * args.steps, launch=launch, graph_ms=graph_ms,
                    graph_substeps=graph_sub, model=model, learn=learn, fallbacks=fallbacks, adaptive=adaptive)


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


def whole_job_rates(times_ms, work, world, device):
    """Whole-job throughput of every leg: the work of all ranks over the slowest
    rank's time (max over ranks of the time, sum over ranks of the work).  Returns
    (rates, (times, work)) with the reduced values."""
    import torch
    t = torch.tensor(times_ms, dtype=torch.float64, device=device)
    w = torch.tensor(work, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(w, op=torch.distributed.ReduceOp.SUM)
    t, w = t.cpu().numpy(), w.cpu().numpy()
    return [float(wi / (ti * 1e-3)) for ti, wi in zip(t, w)], (t, w)


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def reference_arm(args):
    import oracle
    oracle.build.build()
    t_all, cs_all = 0.0, 0
    cores = os.cpu_count() or 1
    for s in range(args.warmup + args.steps):
        v, cores, cs, tt = cpu_baseline_sample(256, seed=100 + s)
        if s >= args.warmup:
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


def extras(b, args):
    """Rows of the batched form beside the headline, each measured once on the GPU:
    the first-order IMEX-MRI step of the 32^3 box captured in a CUDA graph (fast
    stage plus the implicit diffusion solve), the Jacobi-PCG diffusion solve alone
    against the HBM roofline, and the mixed 9/40/80-species reactor batch in one
    launch."""
    import torch

    import mechgen
    mri, w, dev, st = b.mri, b.w, b.dev, b.stream
    out = {}
    hbm = measured_hbm_gbs()

    def timed(fn, reps):
        evs = []
        with torch.cuda.stream(st):
            for _ in range(reps):
                b.flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in evs]

    # IMEX-MRI step (graph-captured; the CG runs a fixed iteration cap without host checks)
    n, ncell = b.n, b.ncell
    y0 = torch.tensor(w.y0, device=dev)
    o = b.opts(1)
    with torch.cuda.stream(st):
        for s in range(2):                       # past the start-up transient, as the MRI steps are
            b.step(y0, 1, s == 0, None)
    torch.cuda.synchronize()
    ws = torch.empty(mri.mri_step_imex1_workspace_size(b.grid, n), dtype=torch.uint8, device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    ss = torch.zeros((ncell, 4), dtype=torch.int32, device=dev)
    y = y0.clone()
    graph = torch.cuda.CUDAGraph()
    st.synchronize()
    with torch.cuda.graph(graph, stream=st):
        mri.mri_step_imex1(y, b.p, b.grid, 0.0, w.H, w.h, b.mech, o, ws, cg_tol=1e-12, cg_max_iter=20,
                           cg_check_every=0, cell_stats=ss, cg_info=info, stream=st)
    y.copy_(y0)
    timed(graph.replay, 2)
    ss.zero_()
    ms = timed(graph.replay, 3)
    sub = int(ss[:, 0].sum().item())
    out["imex1_step"] = {
        "what": "first-order IMEX-MRI step of the 32^3 box (fast stage over H with the explicit advection "
                "plus diffusion forcing, then the implicit diffusion correction by Jacobi-PCG), mixed form, "
                "captured once in a CUDA graph and replayed",
        "ms_per_step": sum(ms) / len(ms), "cell_steps_per_s": sub / (sum(ms) * 1e-3),
        "cg_converged": bool(info[0].item()), "cg_iterations": int(info[1].item())}
    del graph

    # second-order Strang-split IMEX step (Crank-Nicolson half steps around the MRI3 step)
    ws2 = torch.empty(mri.mri_step_imex2_workspace_size(b.grid, n), dtype=torch.uint8, device=dev)
    y.copy_(y0)
    ss.zero_()

    def imex2():
        mri.mri_step_imex2(y, b.p, b.grid, 0.0, w.H, w.h, b.mech, o, ws2, cg_tol=1e-12, cg_max_iter=20,
                           cg_check_every=0, cell_stats=ss, cg_info=info, stream=st)
    timed(imex2, 1)
    ss.zero_()
    ms = timed(imex2, 3)
    sub = int(ss[:, 0].sum().item())
    out["imex2_step"] = {
        "what": "second-order Strang-split IMEX step of the 32^3 box (Crank-Nicolson half steps of the diffusion "
                "by Jacobi-PCG around the MRI3 step with explicit advection), mixed form",
        "ms_per_step": sum(ms) / len(ms), "cell_steps_per_s": sub / (sum(ms) * 1e-3),
        "cg_converged": bool(info[0].item()), "cg_iterations_last_half_step": int(info[1].item())}

    # Jacobi-PCG diffusion solve alone: (I - a D lap_h) x = b on the box's state with
    # a D / dx^2 = 1, iterations fixed at the converged count, against the HBM roofline
    g = w.grid
    a = g["dx"] ** 2 / g["D"]
    rhs = y0.clone()
    x = rhs.clone()
    cws = torch.empty(mri.mri_diffusion_workspace_size(b.grid, n), dtype=torch.uint8, device=dev)
    its = mri.mri_diffusion_solve(x, rhs, b.grid, a, cws, tol=1e-12, max_iter=500, check_every=1, stream=st)
    nbytes = ncell * n * 8

    def solve():
        x.copy_(rhs)
        mri.mri_diffusion_solve(x, rhs, b.grid, a, cws, tol=1e-12, max_iter=its, check_every=0, stream=st)
    timed(solve, 2)
    ms_direct = timed(solve, 5)
    # the same solve recorded once in a CUDA graph (no per-launch host overhead)
    cg_graph = torch.cuda.CUDAGraph()
    st.synchronize()
    with torch.cuda.graph(cg_graph, stream=st):
        solve()
    timed(cg_graph.replay, 2)
    ms = timed(cg_graph.replay, 5)
    del cg_graph
    avg = sum(ms) / len(ms)
    traffic = nbytes * (2 + 5 + its * 11)      # copy of x, the start (r = b - A x, p), 11 doubles per iteration
    out["diffusion_cg"] = {
        "what": "mri_diffusion_solve on the 32^3 x 41 state, a D / dx^2 = 1, tol 1e-12, no host checks, "
                "replayed from a CUDA graph (ms_direct: launched call by call)",
        "iterations": its, "ms": avg, "ms_direct": sum(ms_direct) / len(ms_direct),
        "roofline": {"bound": "hbm", "achieved": traffic / (avg * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": traffic / (avg * 1e-3) / 1e9 / hbm if hbm else None,
                     "traffic": None,
                     "basis": "bytes the kernels move as written: 11 doubles per element and iteration (stencil "
                              "with the p.Ap sums 2, x/r update with the r.r sums 6, direction 3) plus the start "
                              "and the copy of x; the 54 MB working set fits in L2, so this is an L2-resident "
                              "solve measured against the HBM peak from MEASURED_PEAKS.json hbm_gbs"}}

    # mixed 9/40/80-species batch of 0-D reactors, one launch
    batch = mechgen.reactor_batch()
    groups, inits = [], []
    for mech, yy, pp in batch.groups:
        groups.append(dict(mech=mri.mri_mech_load(mech.to_blob()), y=torch.tensor(yy, device=dev),
                           p=torch.tensor(pp, device=dev),
                           cell_stats=torch.zeros((yy.shape[0], 4), dtype=torch.int32, device=dev)))
        inits.append(torch.tensor(yy, device=dev))
    res = {}
    for prec in (0, 1):
        bo = mri.mri_fast_opts_default(method=batch.method, newton_rtol=batch.newton_rtol, ramp=batch.ramp,
                                       jac_policy=mri.MRI_JAC_LAZY, precision=prec)

        def launch():
            for gg, yi in zip(groups, inits):
                gg["y"].copy_(yi)
            mri.mri_stage_fast_batch(groups, 0.0, batch.Hstage, batch.h, bo, stream=st)
        timed(launch, 1)
        for gg in groups:
            gg["cell_stats"].zero_()
        ms = timed(launch, 3)
        sub = sum(int(gg["cell_stats"][:, 0].sum().item()) for gg in groups)
        res[FORMS[prec].split(":")[0]] = {"ms_per_launch": sum(ms) / len(ms), "cell_steps_per_s": sub / (sum(ms) * 1e-3)}
    out["reactor_batch"] = {"what": "4096 constant-pressure 0-D reactors on 9/40/80-species mechanisms "
                                    "(21/170/350 reactions) in one mri_stage_fast_batch launch, one stage of "
                                    "1e-7 s with h = 1e-8 s and the start-up ramp", **res}
    return out


def measured_hbm_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4096, help="cells of the oracle's CPU baseline sample")
    ap.add_argument("--cells-per-side", type=int, default=None,
                    help="shrink the box (profiling captures only; the bench line is for 32^3)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline and the gate (profiling captures)")
    ap.add_argument("--jac", type=int, default=1, help="Newton matrix policy: 0 per substep, 1 lazy")
    ap.add_argument("--tuned-newton-safety", type=float, default=3e-2,
                    help="mri_fast_opts.newton_safety of the tuned forms (the plain form keeps 3e-4)")
    ap.add_argument("--prec", type=int, default=None,
                    help="time one form only: 0 plain FP64, 1 mixed precision, 2 learned start (mixed)")
    ap.add_argument("--no-learned", dest="learned", action="store_false", help="skip the learned form")
    ap.add_argument("--no-adaptive", dest="adaptive", action="store_false",
                    help="skip the adaptive-substep timing of each form")
    ap.add_argument("--no-matrix-cache", dest="matrix_cache", action="store_false",
                    help="refactorise the Newton matrix at the start of every stage instead of keeping it")
    ap.add_argument("--learn-steps", type=int, default=3, help="MRI steps of training data for the learned form")
    ap.add_argument("--learn-epochs", type=int, default=40, help="training epochs of the learned form")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the automatic launch shape instead of timing the candidates")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="skip the CUDA-graph replay of the step")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the IMEX step, diffusion-solve and reactor-batch measurements")
    args = ap.parse_args()
    rank, world = dist_init(args)

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import torch
    b = Bench(args, world)
    forms = [args.prec] if args.prec is not None else ([0, 1, 2] if args.learned else [0, 1])
    results = {}
    for prec in forms:
        r = b.run_form(prec)
        (r["value"], r["e2e_value"]), _ = whole_job_rates([r["total_ms"], r["e2e_ms"]],
                                                          [r["substeps"], r["e2e_substeps"]], world, "cuda")
        r["gate"] = None if (args.no_cpu or rank != 0) else b.gate(r["prec"], r["model"])
        r["model"] = None
        results[prec] = r
    ext = extras(b, args) if args.extras else None
    if rank != 0:
        return
    ok = [p for p in forms if results[p]["gate"] is None or results[p]["gate"]["passed"]]
    head = max(ok, key=lambda p: results[p]["value"]) if ok else forms[0]
    r = results[head]
    peak = b.fp64_peak_tflops

    def roofline(r):
        # dominant kernel (the fast stage): algorithmic FP64 flops per launch over its
        # average event-timed duration, against the measured FP64 FMA pipe rate
        per_launch = r["flops64"] / r["stage_launches"]
        avg_s = r["stage_total_ms"] * 1e-3 / r["stage_launches"]
        ach = per_launch / avg_s / 1e12
        per_cell = STAGE_DRAM_BYTES_PER_CELL.get(r["prec"]) if args.matrix_cache and args.jac == 1 else None
        traffic = None if per_cell is None else per_cell * b.ncell
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch (DRAM read + write)",
                "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 4096-cell launch, "
                                 "scaled to the launch's cells",
                "kernel": "stage_fast_kernel", "fp64_flops_per_launch": per_launch,
                "fp32_flops_per_launch": r["flops32"] / r["stage_launches"], "avg_launch_ms": avg_s * 1e3,
                "peak_basis": "FP64 FMA pipe rate measured in this run (mri_probe_fp64_fma; the pipe issues 2 "
                              "DFMA/clk/SM, %.4f TFLOP/s at 2070 MHz); MEASURED_PEAKS.json has no FP64 entry"
                              % FP64_PEAK_TFLOPS_NOMINAL}

    if args.no_cpu:
        cpu = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": "skipped (--no-cpu)"}
    else:
        cpu_v, cores, cs, tt = cpu_baseline_sample(args.cpu_sample)
        cpu = {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the three fast stages of one MRI step on {args.cpu_sample} sampled cells ({cs} "
                         f"cell-steps, {tt:.1f} s), forcing from the oracle's slow stencil, after an untimed "
                         f"start-up stage"}
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {0: "f64", 1: "f64+f32", 2: "f64+f32+bf16"}[head], "data": "synthetic",
        "config": {"workload": "box32: 32^3 periodic box, 40 species / 170 reactions (12 third-body, 8 Troe), "
                               "MRI3 (Knoth-Wolke MIS) + SDIRK3 fast, H = 5e-8 s, h = H/10, Newton rtol 1e-10, "
                               "4th-order slow stencil; one step = one MRI slow step",
                   "cells": b.ncell, "unknowns_per_cell": b.n, "form": FORMS[head],
                   "jac_policy": ["per-substep", "lazy"][args.jac] + (" + matrix cache across calls"
                                                                      if args.matrix_cache and args.jac == 1
                                                                      else ""),
                   "reduced_for_profiling": args.cells_per_side is not None,
                   "l2": "256 MB buffer written between timed steps",
                   "launch": r["launch"],
                   "newton_per_substep": r["newton"] / max(r["substeps"], 1),
                   "jac_per_substep": r["njac"] / max(r["substeps"], 1), "failed_cells": r["failed"]},
        "clocks": r["clocks"],
        "roofline": roofline(r),
        "cpu_baseline": cpu,
        "e2e": {"value": r["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": (b.ncell * b.n + b.ncell) * 8,
                "d2h_bytes_per_step": b.ncell * b.n * 8},
        "gpu_launches": r["launches"],
        "gate": r["gate"],
        "forms": {FORMS[p]: {"value": results[p]["value"], "e2e": results[p]["e2e_value"],
                             "roofline_frac": roofline(results[p])["frac"], "gate": results[p]["gate"],
                             "newton_per_substep": results[p]["newton"] / max(results[p]["substeps"], 1),
                             "newton_safety": b.newton_safety(results[p]["prec"]),
                             "fast_stage_cell_steps_per_s": results[p]["substeps"] / (results[p]["stage_total_ms"]
                                                                                      * 1e-3),
                             "jac_per_substep": results[p]["njac"] / max(results[p]["substeps"], 1),
                             "launch": results[p]["launch"] and {k: v for k, v in results[p]["launch"].items()
                                                                 if k != "autotuned"},
                             "adaptive_substeps": results[p]["adaptive"],
                             "learned": results[p]["learn"] and dict(
                                 results[p]["learn"], newton_fallbacks=results[p]["fallbacks"],
                                 accept_rate=1.0 - results[p]["fallbacks"] / max(3 * results[p]["substeps"], 1)),
                             "cuda_graph": None if results[p]["graph_ms"] is None else {
                                 "value": results[p]["graph_substeps"] / (results[p]["graph_ms"] * 1e-3),
                                 "ms_per_step": results[p]["graph_ms"] / args.steps,
                                 "note": "the same MRI step (9 kernels, 3 queue resets) captured once and "
                                         "replayed; device-timed like value"},
                             "clocks": results[p]["clocks"]} for p in forms},
    }
    if ext is not None:
        line["extras"] = ext
    print(json.dumps(line))


if __name__ == "__main__":
    main()
