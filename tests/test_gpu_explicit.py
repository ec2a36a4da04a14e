"""The paper's explicit fast methods (Heun, Kutta's third-order method, classical RK4;
Sec. 3.2's MRI-P(k) fast integrators) on the GPU against the oracle: stages with
polynomial forcing on relaxed cells of the 9-species line, with and without the
start-up sequence, whole MRI steps, exact quadrature without chemistry, and the
counters (right-hand-side evaluations, no Jacobian)."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity
from test_oracle_integrators import no_chemistry

pytestmark = pytest.mark.gpu
ORDER = {12: 2, 13: 3, 14: 4}


def relaxed_line(orc):
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    y, st, _ = m.stage_fast(w.y0, w.p, None, w.H, w.h, orc.opts(method=3, ramp=w.ramp))
    assert np.all(st == 0)
    return w, m, y


def gpu_stage(mri, mech, y, p, phi, Hs, h, opts):
    import torch
    gm = mri.mri_mech_load(mech.to_blob())
    yd, pd = torch.tensor(y, device="cuda"), torch.tensor(p, device="cuda")
    ph = None if phi is None else torch.tensor(phi, device="cuda")
    st = torch.full((y.shape[0],), -9, dtype=torch.int32, device="cuda")
    ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, Hs, h, gm, opts, cell_status=st, cell_stats=ss)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy()


@pytest.mark.parametrize("method", [12, 13, 14])
@pytest.mark.parametrize("K,ramp", [(1, 0), (2, 0), (2, 4)])
def test_explicit_stage_matches_oracle(mri, orc, method, K, ramp):
    w, m, y = relaxed_line(orc)
    phi = mechgen.random_forcing(11 + K, y.shape[0], w.mech.n, K)
    Hs = 4e-6
    h = Hs / 32
    ref, rst, rss = m.stage_fast(y, w.p, phi, Hs, h, orc.opts(method=method, ramp=ramp))
    got, gst, gss = gpu_stage(mri, w.mech, y, w.p, phi, Hs, h, mri.mri_fast_opts_default(method=method, ramp=ramp))
    assert np.all(rst == 0) and np.all(gst == 0)
    np.testing.assert_array_equal(gss[:, 0], 32 + ramp)
    np.testing.assert_array_equal(gss[:, 1], (32 + ramp) * ORDER[method])
    np.testing.assert_array_equal(gss[:, 2], 0)
    np.testing.assert_array_equal(gss, rss)
    assert_parity(got, ref, what=f"explicit method {method}, K {K}, ramp {ramp}")


@pytest.mark.parametrize("method", [12, 13, 14])
def test_explicit_stage_without_chemistry_is_exact_quadrature(mri, method):
    rng = np.random.default_rng(method)
    ncell, K = 40, 2
    y = np.concatenate([rng.dirichlet(np.ones(3), ncell), rng.uniform(500, 2000, (ncell, 1))], 1)
    phi = rng.standard_normal((ncell, K, 4)) * np.array([1e3, 1e3, 1e3, 1e7])
    Hs = 3e-8
    got, st, ss = gpu_stage(mri, no_chemistry(), y, np.full(ncell, 101325.0), phi, Hs, 1e-9,
                            mri.mri_fast_opts_default(method=method))
    assert np.all(st == 0)
    expect = y + Hs * sum(phi[:, k, :] / (k + 1) for k in range(K))
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("method", [12, 14])
def test_explicit_mri_step_matches_oracle(mri, orc, method):
    """Two whole MRI3 steps of the relaxed line with an explicit fast method (h = H/100)."""
    import torch
    w, m, y0 = relaxed_line(orc)
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    ref = y0
    for _ in range(2):
        ref, st, _ = m.mri_step(ref, w.p, g, w.H, w.h, orc.opts(method=method))
        assert np.all(st == 0)
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.tensor(y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    ws = torch.empty(mri.mri_step_workspace_size(grid, w.mech.n), dtype=torch.uint8, device="cuda")
    st = torch.zeros(y0.shape[0], dtype=torch.int32, device="cuda")
    for s in range(2):
        mri.mri_step(y, p, grid, s * w.H, w.H, w.h, gm, mri.mri_fast_opts_default(method=method), ws, cell_status=st)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0
    assert_parity(y.cpu().numpy(), ref, what=f"MRI3 with explicit fast method {method}")


def test_explicit_methods_are_rejected_where_they_do_not_apply(mri):
    import torch
    w = mechgen.workload("line64")
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    o = mri.mri_fast_opts_default(method=mri.MRI_ERK4)
    with pytest.raises(mri.MriError):
        mri.mri_stage_fast_guided(y, p, None, 0.0, w.H, w.h, gm, o)
    with pytest.raises(mri.MriError):
        mri.mri_stage_fast_batch([dict(mech=gm, y=y, p=p)], 0.0, w.H, w.h, o)
    with pytest.raises(mri.MriError):
        mri.mri_stage_fast(y, p, None, 0.0, w.H, w.h, gm, mri.mri_fast_opts_default(method=mri.MRI_ERK4, adaptive=1))
