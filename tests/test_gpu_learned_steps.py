"""The learned form's substep-size predictor (learned.LearnedSteps) on the
40-species box at 16^3 cells.  Trained on the accepted step counts of adaptive
solves of the first fast stage of four initial fields (same mechanism), it predicts
each cell's first-step exponent for a fifth, held-out field.  The adaptive stage
started from those steps must match the oracle started from the same steps (the
controller takes the same decisions on both sides), and it must need fewer Newton
iterations, rejected attempts included, than the uniform start.  The first stage
from an initial field takes hundreds of adaptive steps per cell; both sides solve
the stage equations to 1e-11 so that the comparison measures the implementations
rather than where Newton stopped over that many steps."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def test_step_predictor_saves_attempts_and_keeps_parity(mri, orc):
    import torch
    from paper_2211_03293_gb300.learned import LearnedSteps, n_substeps
    w = mechgen.workload("box32", cells_per_side=16)
    n, side = w.mech.n, 16
    gm = mri.mri_mech_load(w.mech.to_blob())
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    ctrl = dict(adaptive=1, ctrl_rtol=1e-6, ctrl_atol_Y=1e-12, ctrl_atol_T=1e-6)
    rtol = 1e-11
    opts = mri.mri_fast_opts_default(method=3, jac_policy=mri.MRI_JAC_LAZY, newton_rtol=rtol, **ctrl)
    Hs = w.H / 3

    def stage_inputs(seed):
        y0, p0 = mechgen.field_3d_hotspots(4000 + seed, side, side, side, w.mech.n_species, g["dx"])
        y = torch.tensor(y0, device="cuda")
        p = torch.tensor(p0, device="cuda")
        fS = torch.empty_like(y)
        mri.mri_slow_rhs(y, fS, grid)
        return y, p, fS[:, None, :].contiguous()

    def adaptive(y, p, phi, k=None):
        yy = y.clone()
        ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
        st = torch.zeros(y.shape[0], dtype=torch.int32, device="cuda")
        mri.mri_stage_fast_guided(yy, p, phi, 0.0, Hs, w.h, gm, opts, cell_status=st, cell_stats=ss, step_exp=k)
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        return yy, ss.cpu().numpy()

    model = LearnedSteps(n, batch=4096)
    for seed in range(1, 5):
        y, p, phi = stage_inputs(seed)
        _, ss = adaptive(y, p, phi)
        model.add(y, p, phi, Hs, w.h, ss[:, 0])
    hist = model.fit(epochs=80, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0], hist

    y, p, phi = stage_inputs(5)
    k = model.step_exp(y, p, phi, Hs)
    out_u, ss_u = adaptive(y, p, phi)
    out_k, ss_k = adaptive(y, p, phi, k)
    kk = k.cpu().numpy()
    k_true = np.log2(n_substeps(Hs, w.h) / np.maximum(ss_u[:, 0], 1))
    err = np.abs(kk - k_true)
    print(f"first-step exponent: predicted mean {kk.mean():.2f} (min {kk.min()}, max {kk.max()}), "
          f"|error| mean {err.mean():.2f}; Newton iterations incl. rejected attempts: uniform start "
          f"{ss_u[:, 1].sum()}, predicted start {ss_k[:, 1].sum()}; accepted steps {ss_u[:, 0].sum()} -> "
          f"{ss_k[:, 0].sum()}")
    assert err.mean() < 1.5
    assert ss_k[:, 1].sum() < ss_u[:, 1].sum()

    # the same first steps on the oracle: the same decisions and the same states
    idx = np.sort(np.random.default_rng(3).choice(y.shape[0], 24, replace=False))
    ref, rst, rss = orc.Mech(w.mech).stage_fast(y.cpu().numpy()[idx], p.cpu().numpy()[idx],
                                                phi.cpu().numpy()[idx], Hs, w.h, orc.opts(method=3, rtol=rtol, **ctrl),
                                                step_exp=kk[idx])
    assert np.all(rst == 0)
    same = ss_k[idx, 0] == rss[:, 0]
    assert same.mean() >= 0.9, (ss_k[idx, 0], rss[:, 0])
    assert_parity(out_k.cpu().numpy()[idx][same], ref[same], what="predicted first steps vs oracle")
    # every sampled cell, those on another step sequence included, against a 100 times
    # tighter oracle solution, within the controller's tolerance
    from test_gpu_adaptive import check_against_tight_solution
    yi, pi, phii = y.cpu().numpy()[idx], p.cpu().numpy()[idx], phi.cpu().numpy()[idx]
    check_against_tight_solution(orc, w, out_k.cpu().numpy()[idx], yi, pi, phii, Hs, ctrl["ctrl_rtol"],
                                 step_exp=kk[idx])
