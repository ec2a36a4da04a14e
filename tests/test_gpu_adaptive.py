"""Adaptive substeps on the GPU (mri_fast_opts.adaptive) against the oracle's
adaptive stage: the power-of-two controller makes the same accept / reject
decisions on both sides, so the accepted step counts agree and the results
match to the Newton tolerance; sampled cells of a full-size 32^3 stage from the
far-from-equilibrium initial state, and relaxed cells at two tolerances."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def run_gpu(mri, w, y, p, phi, Hs, opts):
    import torch
    gm = mri.mri_mech_load(w.mech.to_blob())
    yd, pd = torch.tensor(y, device="cuda"), torch.tensor(p, device="cuda")
    ph = None if phi is None else torch.tensor(phi, device="cuda")
    st = torch.zeros(y.shape[0], dtype=torch.int32, device="cuda")
    ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, Hs, w.h, gm, opts, cell_status=st, cell_stats=ss)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy()


def ctrl(tol):
    return dict(adaptive=1, ctrl_rtol=tol, ctrl_atol_Y=tol * 1e-6, ctrl_atol_T=tol)


@pytest.mark.parametrize("tol", [1e-5, 1e-7])
@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_stage_matches_oracle_on_relaxed_cells(mri, orc, tol, prec):
    w = mechgen.workload("box32")
    m = orc.Mech(w.mech)
    idx = np.sort(np.random.default_rng(5).choice(w.y0.shape[0], 64, replace=False))
    y, p = w.y0[idx], w.p[idx]
    y, st, _ = m.stage_fast(y, p, None, w.H / 3, w.h, orc.opts(method=3, ramp=w.ramp))
    y, st2, _ = m.stage_fast(y, p, None, w.H * 5 / 12, w.h, orc.opts(method=3))
    assert np.all(st == 0) and np.all(st2 == 0)
    phi = mechgen.random_forcing(7, y.shape[0], w.mech.n, 1)
    got, gst, gss = run_gpu(mri, w, y, p, phi, w.H / 4,
                            mri.mri_fast_opts_default(method=3, jac_policy=1, precision=prec, **ctrl(tol)))
    ref, rst, rss = m.stage_fast(y, p, phi, w.H / 4, w.h, orc.opts(method=3, **ctrl(tol)))
    assert np.all(gst == 0) and np.all(rst == 0)
    np.testing.assert_array_equal(gss[:, 0], rss[:, 0])      # the same accepted steps
    assert_parity(got, ref, what=f"adaptive stage tol {tol} form {prec}")


def test_adaptive_full_size_first_stage_sampled(mri, orc):
    """The whole 32^3 box from its initial state (no start-up ramp: the controller
    shrinks the first steps itself), sampled cells against the oracle."""
    w = mechgen.workload("box32")
    fS = orc.slow_rhs(w.y0, w.grid)
    phi = np.ascontiguousarray(fS[:, None, :])
    got, st, ss = run_gpu(mri, w, w.y0, w.p, phi, w.H / 3,
                          mri.mri_fast_opts_default(method=3, jac_policy=1, **ctrl(1e-6)))
    assert int((st != 0).sum()) == 0
    idx = np.sort(np.random.default_rng(8).choice(w.y0.shape[0], 32, replace=False))
    ref, rst, rss = orc.Mech(w.mech).stage_fast(w.y0[idx], w.p[idx], phi[idx], w.H / 3, w.h,
                                                orc.opts(method=3, **ctrl(1e-6)))
    assert np.all(rst == 0)
    same = ss[idx, 0] == rss[:, 0]
    assert same.mean() >= 0.9, (ss[idx, 0], rss[:, 0])
    assert_parity(got[idx][same], ref[same], what="adaptive 32^3 first stage (sampled)")
    # every sampled cell, including those whose controller took another path (an estimate
    # within rounding of a threshold), against a solution 100 times tighter, within the
    # controller's tolerance
    check_against_tight_solution(orc, w, got[idx], w.y0[idx], w.p[idx], phi[idx], w.H / 3, 1e-6)
    print("accepted steps per cell: min", ss[:, 0].min(), "median", np.median(ss[:, 0]), "max", ss[:, 0].max(),
          "; cells on another step sequence:", int((~same).sum()), "of", len(idx))


def check_against_tight_solution(orc, w, got, y, p, phi, Hs, tol, factor=10.0, **kw):
    """Results of cells whose accepted-step sequence differs from the oracle's, against
    the oracle's adaptive solution at a 100 times tighter controller tolerance: the error
    in the controller's own weights (rtol |y| + atol) must stay within factor times its
    tolerance."""
    if got.shape[0] == 0:
        return
    tight, st, _ = orc.Mech(w.mech).stage_fast(y, p, phi, Hs, w.h, orc.opts(method=3, rtol=1e-12,
                                                                               **ctrl(tol / 100.0)), **kw)
    assert np.all(st == 0)
    atol = np.full(got.shape[1], tol * 1e-6)
    atol[-1] = tol
    err = np.abs(got - tight) / (tol * np.abs(tight) + atol)
    assert err.max() <= factor, err.max()
