"""Launch-shape autotuner for mri_stage_fast.

The persistent stage kernel runs one cell per warp; how many warps share a CTA
(and so one staged copy of the mechanism tables) and how many CTAs share an SM
trade shared memory for cells in flight.  The best shape depends on the
mechanism's size, the precision form, K and the cell count, so it is measured:
each candidate shape runs the caller's own stage on a copy of its inputs, timed
with CUDA events on the launching stream, and the fastest is kept.  Every
candidate computes the same result (the launch shape never changes one), so the
tuner needs no checking; the results of the timed runs are discarded.
"""
from . import MriError, mri_fast_opts, mri_stage_fast, mri_stage_fast_shape

_cache = {}


def _with_shape(opts, wpb, bps):
    o = mri_fast_opts.from_buffer_copy(opts)
    o.warps_per_block, o.blocks_per_sm = wpb, bps
    return o


def candidate_shapes(mech, opts, ncell, K, max_bps=4, depth=3):
    """(warps per CTA, CTAs per SM) pairs worth timing: for each CTAs-per-SM count,
    the largest warp count that fits and the next depth-1 below it."""
    out = []
    for bps in range(1, max_bps + 1):
        try:
            wmax, _, _ = mri_stage_fast_shape(mech, _with_shape(opts, 0, bps), 1 << 30, K)
        except MriError:
            continue
        for wpb in range(wmax, max(0, wmax - depth), -1):
            out.append((wpb, bps))
    return out


def autotune_stage(mech, y, p, phi, Hstage, h, opts, repeats=2, stream=None, verbose=False):
    """Time mri_stage_fast over the candidate launch shapes on copies of (y, p, phi)
    and return (opts with the fastest shape, [(wpb, bps, ms), ...]).  The result is
    cached per (mechanism, options, ncell, K, Hstage/h)."""
    import torch
    ncell = y.shape[0]
    K = 0 if phi is None else phi.shape[1]
    key = (id(mech), bytes(opts), ncell, K, round(Hstage / h, 9))
    if key in _cache:
        return _cache[key]
    s = stream or torch.cuda.current_stream()
    work = torch.empty_like(y)
    table = []
    for wpb, bps in candidate_shapes(mech, opts, ncell, K):
        o = _with_shape(opts, wpb, bps)
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
        table.append((wpb, bps, best))
        if verbose:
            print(f"autotune: {wpb} warps/CTA x {bps} CTA/SM: {best:.3f} ms")
    wpb, bps, _ = min(table, key=lambda r: r[2])
    res = (_with_shape(opts, wpb, bps), table)
    _cache[key] = res
    return res
