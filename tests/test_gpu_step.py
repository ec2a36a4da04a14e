"""GPU parity of whole MRI slow steps (mri_step: three f^S evaluations, three
fast stages) against the CPU oracle; at the full 32^3 size, sampled cells of
the first fast stage plus properties that hold at any size."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def gpu_steps(mri, w, nsteps, opts_kw, g=None):
    import torch
    g = g or w.grid
    gm = mri.mri_mech_load(w.mech.to_blob())
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    ws = torch.empty(mri.mri_step_workspace_size(grid, w.mech.n) // 8, dtype=torch.float64, device="cuda")
    st = torch.zeros(w.y0.shape[0], dtype=torch.int32, device="cuda")
    ss = torch.zeros((w.y0.shape[0], 4), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    for s in range(nsteps):
        kw = dict(opts_kw)
        if s > 0:
            kw["ramp"] = 0
        mri.mri_step(y, p, grid, s * w.H, w.H, w.h, gm, mri.mri_fast_opts_default(**kw), ws, cell_status=st,
                     cell_stats=ss, n_failed=nf)
    torch.cuda.synchronize()
    return y.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy(), int(nf.item())


def oracle_steps(orc, w, nsteps, opts_kw, g=None):
    m = orc.Mech(w.mech)
    y = w.y0
    for s in range(nsteps):
        kw = dict(opts_kw)
        if s > 0:
            kw["ramp"] = 0
        y, st, _ = m.mri_step(y, w.p, g or w.grid, w.H, w.h, orc.opts(**kw))
        assert np.all(st == 0)
    return y


def test_mri_step_parity_line64_ten_steps(mri, orc):
    """The whole 64-cell line workload: 10 slow steps of MRI3 with SDIRK2 fast."""
    w = mechgen.workload("line64")
    kw = dict(method=2, ramp=10)
    got, st, ss, nf = gpu_steps(mri, w, w.n_slow_steps, kw)
    ref = oracle_steps(orc, w, w.n_slow_steps, kw)
    assert np.all(st == 0) and nf == 0
    assert np.all(ss[:, 0] == 10 * 101 + 10)
    assert_parity(got, ref, what="line64 10 steps")


@pytest.mark.parametrize("prec", [0, 1])
def test_mri_step_parity_box8(mri, orc, prec):
    """The 40-species box workload at 8^3 cells (ragged against CTA sizes), 2 steps;
    FP64 form and mixed-precision form (FP32 Jacobian / LU, FP64 residual)."""
    w = mechgen.workload("box32", cells_per_side=8)
    kw = dict(method=3, ramp=w.ramp, jac_policy=1, precision=prec)
    got, st, _, nf = gpu_steps(mri, w, 2, kw)
    ref = oracle_steps(orc, w, 2, dict(method=3, ramp=w.ramp))
    assert np.all(st == 0) and nf == 0
    assert_parity(got, ref, what="box 8^3 2 steps")


def test_full_size_box32_first_stage_sampled_and_step_properties(mri, orc):
    """Full 32^3 workload in the launch configuration the bench times: the first
    fast stage of the first step (forcing f^S(y0) from the oracle) compared on 48
    sampled cells, then a whole MRI step checked for properties that hold at any
    size (no failures, sum of Y = 1, grid element totals conserved)."""
    import torch
    w = mechgen.workload("box32")
    n = w.mech.n
    fS = orc.slow_rhs(w.y0, w.grid)           # phi_2 = f^S(Y_1) for the MIS form
    gm = mri.mri_mech_load(w.mech.to_blob())
    yd = torch.tensor(w.y0, device="cuda")
    pd = torch.tensor(w.p, device="cuda")
    ph = torch.tensor(fS[:, None, :].copy(), device="cuda")
    st = torch.zeros(w.y0.shape[0], dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, w.H / 3, w.h, gm,
                       mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=mri.MRI_JAC_LAZY),
                       cell_status=st)
    torch.cuda.synchronize()
    got = yd.cpu().numpy()
    assert int((st != 0).sum()) == 0
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.y0.shape[0], 48, replace=False))
    ref, rst, _ = orc.Mech(w.mech).stage_fast(w.y0[idx], w.p[idx], fS[idx][:, None, :], w.H / 3, w.h,
                                              orc.opts(method=3, ramp=w.ramp))
    assert np.all(rst == 0)
    assert_parity(got[idx], ref, what="32^3 first stage (sampled)")

    out, st, ss, nf = gpu_steps(mri, w, 1, dict(method=3, ramp=w.ramp, jac_policy=mri.MRI_JAC_LAZY))
    assert nf == 0 and np.all(st == 0)
    np.testing.assert_allclose(out[:, :-1].sum(1), 1.0, rtol=0, atol=1e-12)
    E = w.mech.elem / w.mech.W[:, None]
    np.testing.assert_allclose((out[:, :-1] @ E).sum(0), (w.y0[:, :-1] @ E).sum(0), rtol=1e-11)
    assert np.all(ss[:, 0] == (4 + w.ramp) + 5 + 3)


@pytest.mark.parametrize("prec", [0, 1])
def test_matrix_cache_keeps_results_and_saves_jacobians(mri, prec):
    """Three MRI steps of the 8^3 box with the Newton-matrix cache against the same
    steps without it: the same stage solutions (to the Newton tolerance) with fewer
    Jacobian evaluations; an undersized cache is rejected."""
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    kw = dict(method=3, ramp=w.ramp, jac_policy=1, precision=prec)
    plain, st0, ss0, nf0 = gpu_steps(mri, w, 3, kw)
    gm = mri.mri_mech_load(w.mech.to_blob())
    nc = w.y0.shape[0]
    cache = torch.zeros(mri.mri_matrix_cache_size(gm, nc, prec), dtype=torch.uint8, device="cuda")
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    ws = torch.empty(mri.mri_step_workspace_size(grid, w.mech.n) // 8, dtype=torch.float64, device="cuda")
    st = torch.zeros(nc, dtype=torch.int32, device="cuda")
    ss = torch.zeros((nc, 4), dtype=torch.int32, device="cuda")
    for s in range(3):
        o = mri.with_matrix_cache(mri.mri_fast_opts_default(**dict(kw, ramp=kw["ramp"] if s == 0 else 0)), cache)
        mri.mri_step(y, p, grid, s * w.H, w.H, w.h, gm, o, ws, cell_status=st, cell_stats=ss)
    torch.cuda.synchronize()
    got, ss = y.cpu().numpy(), ss.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0) and nf0 == 0
    assert_parity(got, plain, rtol=1e-10, what="matrix cache vs none")
    assert ss[:, 2].sum() < ss0[:, 2].sum()
    assert np.all(ss[:, 0] == ss0[:, 0])
    small = mri.with_matrix_cache(mri.mri_fast_opts_default(**kw), cache[: cache.numel() // 2])
    with pytest.raises(mri.MriError):
        mri.mri_stage_fast(y, p, None, 0.0, w.H / 3, w.h, gm, small)


@pytest.mark.parametrize("prec", [0, 1])
def test_cached_derivative_predicts_the_first_stage(mri, orc, prec):
    """With the matrix cache a call's first SDIRK stage starts from the predictor
    built on f^F kept from the previous call: fewer Newton iterations than the same
    call started from the input state there (the guided start with the input state
    as guess), and both agree with the oracle."""
    import math
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    gm = mri.mri_mech_load(w.mech.to_blob())
    nc, n = w.y0.shape
    kw = dict(method=3, jac_policy=mri.MRI_JAC_LAZY, precision=prec)
    cache = torch.zeros(mri.mri_matrix_cache_size(gm, nc, prec), dtype=torch.uint8, device="cuda")
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    mri.mri_stage_fast(y, p, None, 0.0, w.H / 3, w.h, gm,
                       mri.with_matrix_cache(mri.mri_fast_opts_default(ramp=w.ramp, **kw), cache))
    torch.cuda.synchronize()
    y1 = y.cpu().numpy()
    phi = mechgen.random_forcing(21, nc, n, 1)
    Hs = w.H * 5 / 12
    G = math.ceil(Hs / w.h * (1 - 1e-12))
    ref, rst, _ = orc.Mech(w.mech).stage_fast(y1, w.p, phi, Hs, w.h, orc.opts(method=3))
    assert np.all(rst == 0)
    counts = {}
    for start in (mri.MRI_START_PREDICTOR, mri.MRI_START_GUESS_FIRST):
        yy = torch.tensor(y1, device="cuda")
        c = cache.clone()
        ss = torch.zeros((nc, 4), dtype=torch.int32, device="cuda")
        st = torch.zeros(nc, dtype=torch.int32, device="cuda")
        guess = yy[:, None, :].expand(nc, G, n).contiguous()
        mri.mri_stage_fast_guided(yy, p, torch.tensor(phi, device="cuda"), 0.0, Hs, w.h, gm,
                                  mri.with_matrix_cache(mri.mri_fast_opts_default(**kw), c), start=start,
                                  guess=guess, cell_status=st, cell_stats=ss)
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        assert_parity(yy.cpu().numpy(), ref, what=f"start {start}, form {prec}")
        counts[start] = int(ss[:, 1].sum())
    print(f"form {prec}: Newton iterations with the cached derivative {counts[mri.MRI_START_PREDICTOR]}, "
          f"from the input state {counts[mri.MRI_START_GUESS_FIRST]}")
    assert counts[mri.MRI_START_PREDICTOR] < counts[mri.MRI_START_GUESS_FIRST]
