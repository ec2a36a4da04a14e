"""Learned form end to end on the 40-species box at 16^3 cells: the plain solver
produces substep-end states for the stages of several MRI steps, the network is
trained on them by the library's own kernels, and on held-out stages its
predictions start Newton.  Every result must match the plain solve (same stage
equations, same FP64 acceptance test) and the oracle on sampled cells.  The
network's predictions must beat "no change" by far, and used where the analytic
predictor has no derivative yet (the first SDIRK stage of a call) they must save
Newton iterations there.  Used for every stage instead of the analytic predictor
the network's start costs more iterations than even the previous stage value;
the test prints the counts of all four starts."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def test_learned_start_saves_newton_iterations_and_keeps_parity(mri, orc):
    import torch
    from paper_2211_03293_gb300.learned import LearnedStart, stage_substep_states
    w = mechgen.workload("box32", cells_per_side=16)
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    gm = mri.mri_mech_load(w.mech.to_blob())
    n = w.mech.n
    ncell = w.y0.shape[0]
    c, G = mri.mri_method_coupling(mri.MRI_KW3)
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    fS = torch.empty((3, ncell, n), dtype=torch.float64, device="cuda")
    phi = torch.empty((ncell, 1, n), dtype=torch.float64, device="cuda")
    opts = mri.mri_fast_opts_default(method=3, jac_policy=1)
    model = LearnedStart(n, g_max=5, batch=4096)
    held = []
    for s in range(8):
        for i in range(1, 4):
            mri.mri_slow_rhs(y, fS[i - 1], grid)
            mri.mri_stage_forcing(fS, i, G[i], phi)
            Hs = (c[i] - c[i - 1]) * w.H
            o = mri.mri_fast_opts_default(method=3, jac_policy=1, ramp=w.ramp if (s == 0 and i == 1) else 0)
            y_in = y.clone()
            if s < 6:
                seq, _ = stage_substep_states(y, p, phi, Hs, w.h, gm, o)
                if s > 0:
                    model.add(y_in, p, phi.clone(), Hs, seq)
            else:
                seq, _ = stage_substep_states(y, p, phi, Hs, w.h, gm, o)
                held.append((y_in, phi.clone(), Hs, seq))
    hist = model.fit(epochs=120, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0], hist

    # predictions of the held-out substep-end states beat "no change" by far
    e_net = e_zero = 0.0
    for y_in, ph, Hs, seq in held:
        gss = model.guess(y_in, p, ph, Hs, w.h)
        inc = (seq - y_in[:, None, :]).cpu().numpy()
        e_net += float(np.sum(((gss - seq).cpu().numpy() / (np.abs(inc).max(axis=(0, 1)) + 1e-300)) ** 2))
        e_zero += float(np.sum((inc / (np.abs(inc).max(axis=(0, 1)) + 1e-300)) ** 2))
    print("relative prediction error", np.sqrt(e_net / e_zero))
    assert e_net < 0.25 * e_zero

    totals = {}
    for start in (mri.MRI_START_PREVIOUS, mri.MRI_START_GUESS, mri.MRI_START_PREDICTOR, mri.MRI_START_GUESS_FIRST):
        its, fb, outs = 0, 0, []
        for y_in, ph, Hs, _ in held:
            yy = y_in.clone()
            st = torch.zeros(ncell, dtype=torch.int32, device="cuda")
            ss = torch.zeros((ncell, 4), dtype=torch.int32, device="cuda")
            nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
            guess = model.guess(y_in, p, ph, Hs, w.h) if start in (mri.MRI_START_GUESS,
                                                                    mri.MRI_START_GUESS_FIRST) else None
            mri.mri_stage_fast_guided(yy, p, ph, 0.0, Hs, w.h, gm, opts, start=start, guess=guess, cell_status=st,
                                      cell_stats=ss, n_fallback=nfb)
            torch.cuda.synchronize()
            assert int((st != 0).sum()) == 0
            its += int(ss[:, 1].sum())
            fb += int(nfb.item())
            outs.append(yy.cpu().numpy())
        totals[start] = (its, fb, outs)
    print("Newton iterations and fallbacks per start:", {k: v[:2] for k, v in totals.items()})
    # the network's start where the predictor has nothing to extrapolate from (the
    # first SDIRK stage of each call) saves Newton iterations over the plain start
    # there (the previous stage value); no stage needed the fallback
    assert totals[mri.MRI_START_GUESS_FIRST][0] < totals[mri.MRI_START_PREDICTOR][0]
    assert totals[mri.MRI_START_GUESS_FIRST][1] == 0
    # same stage solutions whatever the start: all within the Newton tolerance
    for start in totals:
        for a, b in zip(totals[start][2], totals[mri.MRI_START_PREDICTOR][2]):
            assert_parity(a, b, rtol=1e-9, what=f"start {start} vs predictor")
    # and the oracle on sampled cells of the first held-out stage, from the network's start
    y_in, ph, Hs, _ = held[0]
    idx = np.sort(np.random.default_rng(0).choice(ncell, 16, replace=False))
    ref, rst, _ = orc.Mech(w.mech).stage_fast(y_in.cpu().numpy()[idx], w.p[idx], ph.cpu().numpy()[idx], Hs, w.h,
                                              orc.opts(method=3))
    assert np.all(rst == 0)
    assert_parity(totals[mri.MRI_START_GUESS][2][0][idx], ref, what="learned start vs oracle")
