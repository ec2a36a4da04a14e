"""GPU parity of one MRI stage of the fast partition (mri_stage_fast) against the
CPU oracle, plus exact reductions, edge cases, failure reporting and
determinism."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def run_gpu(mri, mech_blob, y, p, phi, Hs, h, opts, stats=True):
    import torch
    gm = mri.mri_mech_load(mech_blob)
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    ph = None if phi is None else torch.tensor(phi, dtype=torch.float64, device="cuda")
    st = torch.full((y.shape[0],), -9, dtype=torch.int32, device="cuda")
    ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, Hs, h, gm, opts, cell_status=st, cell_stats=ss if stats else None,
                       n_failed=nf)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy(), int(nf.item())


def sample(w, n, seed):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.y0.shape[0], n, replace=False))
    return w.y0[idx], w.p[idx]


@pytest.mark.parametrize("K,ramp,prec", [(1, 10, 0), (0, 10, 0), (3, 10, 0), (1, 10, 1)])
def test_stage_parity_line64(mri, orc, K, ramp, prec):
    w = mechgen.workload("line64")
    phi = mechgen.random_forcing(5, 64, w.mech.n, K) if K else None
    opts = mri.mri_fast_opts_default(method=2, ramp=ramp, precision=prec)
    got, st, ss, nf = run_gpu(mri, w.mech.to_blob(), w.y0, w.p, phi, w.H / 3, w.h, opts)
    ref, rst, rss = orc.Mech(w.mech).stage_fast(w.y0, w.p, phi, w.H / 3, w.h, orc.opts(method=2, ramp=ramp))
    assert np.all(st == 0) and np.all(rst == 0) and nf == 0
    assert np.all(ss[:, 0] == 34 + ramp) and np.all(ss[:, 3] == 0)
    assert_parity(got, ref, what="line64 stage")


@pytest.mark.parametrize("K,jac,prec", [(0, 0, 0), (2, 0, 0), (2, 1, 0), (2, 1, 1), (0, 0, 1)])
def test_stage_parity_box32_sample(mri, orc, K, jac, prec):
    w = mechgen.workload("box32")
    y, p = sample(w, 301, 3)
    phi = mechgen.random_forcing(6, y.shape[0], w.mech.n, K) if K else None
    opts = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=jac, precision=prec)
    got, st, ss, nf = run_gpu(mri, w.mech.to_blob(), y, p, phi, w.H / 3, w.h, opts)
    ref, rst, _ = orc.Mech(w.mech).stage_fast(y, p, phi, w.H / 3, w.h, orc.opts(method=3, ramp=w.ramp))
    assert np.all(rst == 0)
    assert np.all(st == 0) and nf == 0
    assert np.all(ss[:, 0] == 4 + w.ramp)
    assert_parity(got, ref, what="box32 stage")


@pytest.mark.parametrize("jac,prec", [(0, 0), (1, 0), (1, 1)])
def test_stage_parity_relaxed_state_box32(mri, orc, jac, prec):
    """After the start-up transient (no ramp, the usual Newton count per stage)."""
    w = mechgen.workload("box32")
    y, p = sample(w, 96, 4)
    om = orc.Mech(w.mech)
    y1, rst, _ = om.stage_fast(y, p, None, w.H / 3, w.h, orc.opts(method=3, ramp=w.ramp))
    assert np.all(rst == 0)
    phi = mechgen.random_forcing(8, y.shape[0], w.mech.n, 1)
    opts = mri.mri_fast_opts_default(method=3, jac_policy=jac, precision=prec)
    got, st, ss, _ = run_gpu(mri, w.mech.to_blob(), y1, p, phi, w.H * 5 / 12, w.h, opts)
    ref, rst, _ = om.stage_fast(y1, p, phi, w.H * 5 / 12, w.h, orc.opts(method=3))
    assert np.all(st == 0) and np.all(rst == 0)
    assert_parity(got, ref, what="box32 relaxed stage")


@pytest.mark.parametrize("method,K", [(2, 2), (3, 3)])
def test_stage_without_chemistry_is_exact_quadrature(mri, method, K):
    from test_oracle_integrators import no_chemistry
    mech = no_chemistry()
    rng = np.random.default_rng(K)
    ncell = 40
    y = np.concatenate([rng.dirichlet(np.ones(3), ncell), rng.uniform(500, 2000, (ncell, 1))], 1)
    phi = rng.standard_normal((ncell, K, 4)) * np.array([1e3, 1e3, 1e3, 1e7])
    Hs = 3e-8
    got, st, ss, _ = run_gpu(mri, mech.to_blob(), y, np.full(ncell, 101325.0), phi, Hs, 1e-9,
                             mri.mri_fast_opts_default(method=method, ramp=4))
    expect = y + Hs * sum(phi[:, k, :] / (k + 1) for k in range(K))
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-16)
    assert np.all(ss[:, 0] == 34)


def test_stage_zero_cells(mri):
    import torch
    w = mechgen.workload("line64")
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.zeros((0, w.mech.n), dtype=torch.float64, device="cuda")
    p = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert mri.mri_stage_fast(y, p, None, 0.0, 1e-8, 1e-9, gm, mri.mri_fast_opts_default()) == 0


def test_stage_single_cell_and_max_species(mri, orc):
    """One cell; and a mechanism at the species limit of the kernels (127)."""
    w = mechgen.workload("line64")
    got, st, _, _ = run_gpu(mri, w.mech.to_blob(), w.y0[7:8], w.p[7:8], None, w.H / 4, w.h,
                            mri.mri_fast_opts_default(method=2, ramp=10))
    ref, _, _ = orc.Mech(w.mech).stage_fast(w.y0[7:8], w.p[7:8], None, w.H / 4, w.h, orc.opts(method=2, ramp=10))
    assert_parity(got, ref)
    big = mechgen.make_mechanism(77, n_species=127, n_reactions=150, elements=("C", "H", "O", "N"),
                                 n_thirdbody=3, n_troe=2, max_atoms=7, max_count=[3, 6, 3, 3])
    rng = np.random.default_rng(1)
    y = np.concatenate([rng.dirichlet(np.ones(127), 5), rng.uniform(800, 1500, (5, 1))], 1)
    p = np.full(5, 101325.0)
    got, st, _, _ = run_gpu(mri, big.to_blob(), y, p, None, 1e-9, 2.5e-10,
                            mri.mri_fast_opts_default(method=3, ramp=12, max_newton=30))
    ref, rst, _ = orc.Mech(big).stage_fast(y, p, None, 1e-9, 2.5e-10, orc.opts(method=3, ramp=12, max_newton=30))
    ok = (st == 0) & (rst == 0)
    assert ok.sum() >= 3
    assert_parity(got[ok], ref[ok], what="127 species")


def test_stage_rejects_bad_cell_state(mri):
    w = mechgen.workload("line64")
    y = w.y0[:6].copy()
    y[1, -1] = -5.0            # T <= 0
    y[3, 2] = np.nan           # non-finite mass fraction
    p = w.p[:6].copy()
    p[4] = 0.0                 # p <= 0
    got, st, ss, nf = run_gpu(mri, w.mech.to_blob(), y, p, None, w.H / 4, w.h,
                              mri.mri_fast_opts_default(method=2, ramp=10))
    assert list(st) == [0, 2, 0, 2, 2, 0]
    assert nf == 3
    np.testing.assert_array_equal(got[1], y[1])
    np.testing.assert_array_equal(got[4], y[4])
    assert np.isnan(got[3, 2])


def test_stage_reports_newton_failure(mri, orc):
    """max_newton = 1 cannot converge to 1e-10: every cell fails in its first stage
    and keeps its input state, on both sides."""
    w = mechgen.workload("box32")
    y, p = sample(w, 40, 9)
    got, st, ss, nf = run_gpu(mri, w.mech.to_blob(), y, p, None, w.H / 3, w.h,
                              mri.mri_fast_opts_default(method=3, max_newton=1))
    ref, rst, _ = orc.Mech(w.mech).stage_fast(y, p, None, w.H / 3, w.h, orc.opts(method=3, max_newton=1))
    np.testing.assert_array_equal(st, rst)
    assert np.all(st == 1) and nf == 40
    np.testing.assert_array_equal(got, y)
    assert np.all(ss[:, 3] == 1) and np.all(ss[:, 0] == 0)


def test_stage_is_deterministic(mri):
    w = mechgen.workload("box32")
    y, p = sample(w, 200, 12)
    phi = mechgen.random_forcing(1, 200, w.mech.n, 1)
    opts = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=1)
    a = run_gpu(mri, w.mech.to_blob(), y, p, phi, w.H / 4, w.h, opts)
    b = run_gpu(mri, w.mech.to_blob(), y, p, phi, w.H / 4, w.h, opts)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])
