"""Autotuner for mri_stage_fast.

The persistent stage kernel runs one cell per warp.  Its cost depends on choices
that never change a result:

* cells per CTA and CTAs per SM (``warps_per_block``, ``blocks_per_sm``): how many
  cells share one staged copy of the mechanism tables, traded against the shared
  memory of each cell's workspace;
* the layout of the triangular solves (``lu_variant``): the solution in registers
  with rows lane + 32 r, the split forward layout, or substitutions in shared
  memory;
* the scheduling of cells to warps (``schedule``): the device work queue or the
  static round-robin mapping.

The best choice depends on the mechanism's size, the precision form, K and the
cell count, so it is measured: each candidate runs the caller's own stage on a copy
of its inputs, timed with CUDA events on the launching stream.  The search is
coordinate-wise (launch shapes first, then the solve layout at the best shape, then
the schedule).  Every candidate but the Gauss-Jordan inverse (MRI_LU_INVERSE)
computes the same result bit for bit, and that one differs by rounding inside the
Newton tolerance, so the tuner needs no checking and the results of the timed runs
are discarded.
"""
from . import (MRI_LU_AUTO, MRI_LU_INVERSE, MRI_LU_REGS, MRI_LU_REGS_SPLIT, MRI_LU_SHARED, MRI_SCHED_QUEUE,
               MRI_SCHED_STATIC,
               MriError, mri_fast_opts, mri_stage_fast, mri_stage_fast_shape)

_cache = {}


def _with(opts, **kw):
    o = mri_fast_opts.from_buffer_copy(opts)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def candidate_shapes(mech, opts, ncell, K, max_bps=4, depth=3):
    """(warps per CTA, CTAs per SM) pairs worth timing: for each CTAs-per-SM count,
    the largest warp count that fits and the next depth-1 below it."""
    out = []
    for bps in range(1, max_bps + 1):
        try:
            wmax, _, _ = mri_stage_fast_shape(mech, _with(opts, warps_per_block=0, blocks_per_sm=bps), 1 << 30, K)
        except MriError:
            continue
        for wpb in range(wmax, max(0, wmax - depth), -1):
            out.append((wpb, bps))
    return out


def candidate_lu_variants(n):
    """Factorisations and solve layouts that differ for a system of n unknowns."""
    if n <= 32:
        return [MRI_LU_REGS, MRI_LU_SHARED, MRI_LU_INVERSE]
    if n <= 64:
        return [MRI_LU_REGS, MRI_LU_REGS_SPLIT, MRI_LU_SHARED, MRI_LU_INVERSE]
    return [MRI_LU_SHARED, MRI_LU_INVERSE]


def autotune_stage(mech, y, p, phi, Hstage, h, opts, repeats=2, stream=None, verbose=False, schedules=True):
    """Time mri_stage_fast over the candidates on copies of (y, p, phi) and return
    (opts with the fastest choice, [(wpb, bps, lu_variant, schedule, ms), ...]).
    The result is cached per (mechanism, options, ncell, K, Hstage/h)."""
    import torch
    ncell = y.shape[0]
    K = 0 if phi is None else phi.shape[1]
    key = (id(mech), bytes(opts), ncell, K, round(Hstage / h, 9), schedules)
    if key in _cache:
        return _cache[key]
    s = stream or torch.cuda.current_stream()
    work = torch.empty_like(y)
    table = []

    def timed(o):
        best = None
        for _ in range(repeats):
            work.copy_(y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(s):
                e0.record()
                mri_stage_fast(work, p, phi, 0.0, Hstage, h, mech, o, stream=s)
                e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        table.append((o.warps_per_block, o.blocks_per_sm, o.lu_variant, o.schedule, best))
        if verbose:
            print(f"autotune: {o.warps_per_block} warps/CTA x {o.blocks_per_sm} CTA/SM, solve layout "
                  f"{o.lu_variant}, schedule {o.schedule}: {best:.3f} ms")
        return best

    base = _with(opts, lu_variant=MRI_LU_AUTO, schedule=MRI_SCHED_QUEUE)
    best_o, best_ms = None, None
    for wpb, bps in candidate_shapes(mech, base, ncell, K):
        o = _with(base, warps_per_block=wpb, blocks_per_sm=bps)
        ms = timed(o)
        if best_ms is None or ms < best_ms:
            best_o, best_ms = o, ms
    for v in candidate_lu_variants(mech.n):
        o = _with(best_o, lu_variant=v)
        ms = timed(o)
        if ms < best_ms:
            best_o, best_ms = o, ms
    if schedules and opts.time_budget_s == 0.0:
        o = _with(best_o, schedule=MRI_SCHED_STATIC)
        ms = timed(o)
        if ms < best_ms:
            best_o, best_ms = o, ms
    res = (best_o, table)
    _cache[key] = res
    return res
