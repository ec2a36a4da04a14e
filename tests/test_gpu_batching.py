"""The batched form's machinery: launch shapes of the persistent kernel, its device
work queue (time budget, concurrent launches) and CUDA-graph capture of whole MRI
steps.  None of these may change a result: each case compares bit for bit with a
plain launch, whose parity against the oracle the stage and step tests establish."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def box_sample(n, seed):
    w = mechgen.workload("box32")
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.y0.shape[0], n, replace=False))
    return w, w.y0[idx], w.p[idx]


def launch(mri, gm, y, p, phi, Hs, h, opts, stream=None):
    import torch
    yd = torch.tensor(y, device="cuda")
    pd = torch.tensor(p, device="cuda")
    ph = None if phi is None else torch.tensor(phi, device="cuda")
    st = torch.full((y.shape[0],), -9, dtype=torch.int32, device="cuda")
    ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, Hs, h, gm, opts, cell_status=st, cell_stats=ss, n_failed=nf, stream=stream)
    return yd, st, ss, nf


def host(*ts):
    import torch
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in ts]


@pytest.mark.parametrize("prec", [0, 1])
def test_launch_shape_does_not_change_results(mri, prec):
    w, y, p = box_sample(300, 21)
    phi = mechgen.random_forcing(2, y.shape[0], w.mech.n, 1)
    gm = mri.mri_mech_load(w.mech.to_blob())
    runs = []
    shapes = [dict(warps_per_block=wpb, blocks_per_sm=bps) for wpb, bps in
              [(0, 0), (1, 0), (3, 0), (0, 2), (2, 2), (1, 3)]]
    # the solve layouts and the static schedule change the cost only, never a bit of the result
    shapes += [dict(lu_variant=v) for v in (mri.MRI_LU_REGS, mri.MRI_LU_REGS_SPLIT, mri.MRI_LU_SHARED)]
    shapes += [dict(schedule=mri.MRI_SCHED_STATIC), dict(schedule=mri.MRI_SCHED_STATIC, warps_per_block=2)]
    for kw in shapes:
        o = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=1, precision=prec, **kw)
        runs.append(host(*launch(mri, gm, y, p, phi, w.H / 3, w.h, o)[:3]))
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)
    assert np.all(runs[0][1] == 0)


def test_launch_shape_that_does_not_fit_is_rejected(mri):
    w = mechgen.workload("box32")
    gm = mri.mri_mech_load(w.mech.to_blob())
    y, p = w.y0[:4], w.p[:4]
    # 16 warps of a 40-species workspace do not fit in one SM's shared memory
    with pytest.raises(mri.MriError):
        launch(mri, gm, y, p, None, w.H / 3, w.h, mri.mri_fast_opts_default(warps_per_block=16))


def test_autotuner_picks_a_timed_shape_with_the_same_result(mri):
    import torch
    from paper_2211_03293_gb300.autotune import autotune_stage, candidate_shapes
    w, y, p = box_sample(2000, 24)
    gm = mri.mri_mech_load(w.mech.to_blob())
    o = mri.mri_fast_opts_default(method=3, jac_policy=1, precision=1)
    yd, pd = torch.tensor(y, device="cuda"), torch.tensor(p, device="cuda")
    cands = candidate_shapes(gm, o, y.shape[0], 0)
    assert (mri.mri_stage_fast_shape(gm, o, 1 << 30, 0)[0], 1) in cands
    best, table = autotune_stage(gm, yd, pd, None, w.H / 5, w.h, o, repeats=1)
    # every launch shape, then the three solve layouts and the inverse at the best shape,
    # then the static schedule
    assert len(table) == len(cands) + 4 + 1 and all(r[-1] > 0 for r in table)
    fastest = min(table, key=lambda r: r[-1])
    assert (best.warps_per_block, best.blocks_per_sm, best.lu_variant, best.schedule) == fastest[:4]
    np.testing.assert_array_equal(yd.cpu().numpy(), y)          # the tuner worked on copies
    a = host(launch(mri, gm, y, p, None, w.H / 5, w.h, o)[0])[0]
    b = host(launch(mri, gm, y, p, None, w.H / 5, w.h, best)[0])[0]
    if best.lu_variant == mri.MRI_LU_INVERSE:    # the inverse rounds differently, inside the tolerance
        assert_parity(b, a, what="autotuned (inverse) against the default")
    else:
        np.testing.assert_array_equal(a, b)


def test_time_budget_leaves_a_resumable_tail(mri):
    """A budget (50 us) far shorter than one cell's solve (about 2 ms for this stage
    with its start-up substeps): each warp finishes the cell it took
    first and takes no other.  The cells run are a prefix; the rest keep their state,
    report MRI_CELL_TIMEOUT and are counted as failed; a second call on that tail
    completes the stage with the same result as an unbudgeted call."""
    import torch
    w, y, p = box_sample(4000, 22)
    phi = mechgen.random_forcing(3, y.shape[0], w.mech.n, 1)
    gm = mri.mri_mech_load(w.mech.to_blob())
    base = dict(method=3, ramp=w.ramp, jac_policy=1)
    ref = host(*launch(mri, gm, y, p, phi, w.H / 3, w.h, mri.mri_fast_opts_default(**base))[:3])
    short = mri.mri_fast_opts_default(time_budget_s=5e-5, **base)
    wpb, blocks, _ = mri.mri_stage_fast_shape(gm, short, y.shape[0], 1)
    yd, st, ss, nf = launch(mri, gm, y, p, phi, w.H / 3, w.h, short)
    got, gst, gss, gnf = host(yd, st, ss, nf)
    done = int((gst == mri.MRI_CELL_OK).sum())
    assert 1 <= done <= wpb * blocks < y.shape[0]
    assert np.all(gst[:done] == mri.MRI_CELL_OK) and np.all(gst[done:] == mri.MRI_CELL_TIMEOUT)
    assert int(gnf[0]) == y.shape[0] - done
    np.testing.assert_array_equal(got[:done], ref[0][:done])
    np.testing.assert_array_equal(gss[:done], ref[2][:done])
    np.testing.assert_array_equal(got[done:], y[done:])
    assert np.all(gss[done:] == 0)
    # resume on the tail, in place
    pd = torch.tensor(p, device="cuda")
    ph = torch.tensor(phi, device="cuda")
    st2 = st[done:]
    mri.mri_stage_fast(yd[done:], pd[done:], ph[done:], 0.0, w.H / 3, w.h, gm, mri.mri_fast_opts_default(**base),
                       cell_status=st2, cell_stats=ss[done:])
    got, gst, gss = host(yd, st, ss)
    np.testing.assert_array_equal(got, ref[0])
    np.testing.assert_array_equal(gss, ref[2])
    assert np.all(gst == 0)
    # a generous budget changes nothing
    big = host(*launch(mri, gm, y, p, phi, w.H / 3, w.h, mri.mri_fast_opts_default(time_budget_s=600.0, **base)))
    np.testing.assert_array_equal(big[0], ref[0])
    assert np.all(big[1] == 0) and int(big[3][0]) == 0


def test_concurrent_launches_on_two_streams(mri):
    """Two launches on the same mechanism in flight together on two streams take
    separate queue counters: each matches the same launch run alone."""
    import torch
    w, y, p = box_sample(1200, 23)
    gm = mri.mri_mech_load(w.mech.to_blob())
    o = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=1)
    half = y.shape[0] // 2
    alone_a = host(launch(mri, gm, y[:half], p[:half], None, w.H / 3, w.h, o)[0])[0]
    alone_b = host(launch(mri, gm, y[half:], p[half:], None, w.H / 4, w.h, o)[0])[0]
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    ra = launch(mri, gm, y[:half], p[:half], None, w.H / 3, w.h, o, stream=sa)
    rb = launch(mri, gm, y[half:], p[half:], None, w.H / 4, w.h, o, stream=sb)
    ga, gb = host(ra[0], rb[0])
    np.testing.assert_array_equal(ga, alone_a)
    np.testing.assert_array_equal(gb, alone_b)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_captured_mri_steps_match_eager_steps(mri, prec):
    """Whole MRI steps (slow stencil, forcing, three fast stages and their queue
    resets) recorded once in a CUDA graph and replayed give the eager steps' states,
    statuses and counters bit for bit."""
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    gm = mri.mri_mech_load(w.mech.to_blob())
    nc, n = w.y0.shape
    first = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=1, precision=prec)
    later = mri.mri_fast_opts_default(method=3, jac_policy=1, precision=prec)

    def buffers():
        return (torch.tensor(w.y0, device="cuda"), torch.tensor(w.p, device="cuda"),
                torch.empty(mri.mri_step_workspace_size(grid, n) // 8, dtype=torch.float64, device="cuda"),
                torch.zeros(nc, dtype=torch.int32, device="cuda"),
                torch.zeros((nc, 4), dtype=torch.int32, device="cuda"),
                torch.zeros(1, dtype=torch.int32, device="cuda"))

    def step(b, opts, s):
        y, p, ws, st, ss, nf = b
        mri.mri_step(y, p, grid, s * w.H, w.H, w.h, gm, opts, ws, cell_status=st, cell_stats=ss, n_failed=nf)

    eager = buffers()
    for s in range(4):
        step(eager, first if s == 0 else later, s)
    ref = host(*eager[:1], *eager[3:])

    cap = buffers()
    step(cap, first, 0)          # the start-up step runs eagerly
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(cap, later, 1)
    for _ in range(3):
        graph.replay()
    got = host(*cap[:1], *cap[3:])
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)
    assert int(got[-1][0]) == 0
