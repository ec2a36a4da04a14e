"""Host-side guards of the library on one GPU: every call that uses a mechanism
refuses to run with another device current (checked through a test hook that
records another device on the mechanism), and fast-stage launches recorded in a
CUDA graph keep work-queue counters that eager launches never take, so replays and
eager launches overlapping on two streams both integrate every cell."""
import numpy as np
import pytest

import mechgen

pytestmark = pytest.mark.gpu


def test_calls_with_another_device_current_are_rejected(mri):
    import torch
    w = mechgen.workload("line64")
    gm = mri.mri_mech_load(w.mech.to_blob())
    n, ncell = w.mech.n, w.y0.shape[0]
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    y = torch.tensor(w.y0, device="cuda")
    y_before = y.clone()
    p = torch.tensor(w.p, device="cuda")
    phi = torch.zeros((ncell, 1, n), dtype=torch.float64, device="cuda")
    f = torch.zeros((ncell, n), dtype=torch.float64, device="cuda")
    J = torch.zeros((ncell, n, n), dtype=torch.float64, device="cuda")
    o = mri.mri_fast_opts_default(method=w.method, ramp=w.ramp)
    ws = torch.empty(mri.mri_step_imex2_workspace_size(grid, n), dtype=torch.uint8, device="cuda")
    dev = torch.cuda.current_device()
    calls = {
        "mri_stage_fast": lambda: mri.mri_stage_fast(y, p, phi, 0.0, w.H, w.h, gm, o),
        "mri_stage_fast_guided": lambda: mri.mri_stage_fast_guided(y, p, phi, 0.0, w.H, w.h, gm, o),
        "mri_stage_fast_batch": lambda: mri.mri_stage_fast_batch([dict(mech=gm, y=y, p=p)], 0.0, w.H, w.h, o),
        "mri_step": lambda: mri.mri_step(y, p, grid, 0.0, w.H, w.h, gm, o, ws),
        "mri_step_noalloc": lambda: mri.mri_step_noalloc(y, p, grid, 0.0, w.H, w.h, gm, o),
        "mri_step_imex1": lambda: mri.mri_step_imex1(y, p, grid, 0.0, w.H, w.h, gm, o, ws),
        "mri_step_imex2": lambda: mri.mri_step_imex2(y, p, grid, 0.0, w.H, w.h, gm, o, ws),
        "mri_fast_rhs": lambda: mri.mri_fast_rhs(y, p, gm, f),
        "mri_fast_jac": lambda: mri.mri_fast_jac(y, p, gm, J),
    }
    torch.cuda.synchronize()
    assert mri.mri_probe_mech_device(gm, dev + 1) == dev
    try:
        for name, call in calls.items():
            with pytest.raises(mri.MriError) as e:
                call()
            assert e.value.code == mri.MRI_EINVAL, name
    finally:
        assert mri.mri_probe_mech_device(gm, dev) == dev + 1
    torch.cuda.synchronize()
    assert torch.equal(y, y_before)                  # nothing was launched
    mri.mri_stage_fast(y, p, phi, 0.0, w.H, w.h, gm, o)
    torch.cuda.synchronize()
    assert not torch.equal(y, y_before)


def test_graph_replays_and_eager_launches_keep_their_own_queue_counters(mri):
    """A graph with one captured stage launch is replayed on one stream while more
    eager launches than the eager ring holds run on another: both results equal the
    same launches run alone."""
    import torch
    w = mechgen.workload("line64")
    gm = mri.mri_mech_load(w.mech.to_blob())
    n = w.mech.n
    rng = np.random.default_rng(4)
    o = mri.mri_fast_opts_default(method=w.method, ramp=w.ramp)
    # the graph's cells (all 64) and a small eager batch
    yg0 = torch.tensor(w.y0, device="cuda")
    pg = torch.tensor(w.p, device="cuda")
    ye0 = torch.tensor(w.y0[rng.choice(w.y0.shape[0], 4, replace=False)], device="cuda")
    pe = torch.tensor(np.full(4, 101325.0), device="cuda")
    Hs = w.H / 3
    ref_g = yg0.clone()
    ref_e = ye0.clone()
    mri.mri_stage_fast(ref_g, pg, None, 0.0, Hs, w.h, gm, o)
    mri.mri_stage_fast(ref_e, pe, None, 0.0, Hs, w.h, gm, o)
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    yg = yg0.clone()
    graph = torch.cuda.CUDAGraph()
    sa.synchronize()
    with torch.cuda.graph(graph, stream=sa):
        yg.copy_(yg0)
        mri.mri_stage_fast(yg, pg, None, 0.0, Hs, w.h, gm, o, stream=sa)
    torch.cuda.synchronize()
    outs = [torch.empty_like(ye0) for _ in range(300)]
    with torch.cuda.stream(sb):
        for k in range(300):
            outs[k].copy_(ye0)
            mri.mri_stage_fast(outs[k], pe, None, 0.0, Hs, w.h, gm, o, stream=sb)
            if k % 20 == 0:
                with torch.cuda.stream(sa):
                    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(yg, ref_g)
    for k in range(300):
        assert torch.equal(outs[k], ref_e), k
    del graph
