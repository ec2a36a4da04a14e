"""Pins of the oracle's adaptive fast stage (substep sizes from an embedded error
estimate): the embedded weights' order conditions, exact quadrature of the
forcing whatever the step sequence, convergence to a fine fixed-step solution as
the controller's tolerance shrinks, and far fewer steps on quiet cells."""
import numpy as np
import pytest

import mechgen
from test_oracle_integrators import no_chemistry


@pytest.mark.parametrize("method", [2, 3])
def test_embedded_weights_order_conditions(orc, method):
    A, b, c = orc.sdirk_tableau(method)
    bhat, q = orc.sdirk_embedded(method)
    assert abs(bhat.sum() - 1.0) < 1e-15                      # consistency
    if method == 3:
        assert abs(bhat @ c - 0.5) < 1e-15                    # second order
        assert abs((b - bhat) @ c ** 2) > 1e-3                # the estimate's leading term is O(h^3)
        assert q == 3
    else:
        assert abs((b - bhat) @ c) > 1e-3                     # O(h^2)
        assert q == 2


@pytest.mark.parametrize("method,K", [(2, 2), (3, 3)])
def test_adaptive_stage_without_chemistry_is_exact_quadrature(orc, method, K):
    mech = no_chemistry()
    m = orc.Mech(mech)
    rng = np.random.default_rng(10 + K)
    ncell = 6
    y = np.concatenate([rng.dirichlet(np.ones(3), ncell), rng.uniform(500, 2000, (ncell, 1))], 1)
    phi = rng.standard_normal((ncell, K, 4)) * np.array([1e3, 1e3, 1e3, 1e7])
    Hs = 3e-8
    out, st, ss = m.stage_fast(y, np.full(ncell, 101325.0), phi, Hs, 1e-9,
                               orc.opts(method=method, adaptive=1, ctrl_rtol=1e-9, ctrl_atol_Y=1e-14,
                                        ctrl_atol_T=1e-9))
    assert np.all(st == 0)
    expect = y + Hs * sum(phi[:, k, :] / (k + 1) for k in range(K))
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-16)


def _relaxed_box_cells(orc, n=12, seed=1):
    """Box cells after two fast stages (past the start-up transient)."""
    w = mechgen.workload("box32")
    m = orc.Mech(w.mech)
    idx = np.sort(np.random.default_rng(seed).choice(w.y0.shape[0], n, replace=False))
    y, p = w.y0[idx], w.p[idx]
    y, st, _ = m.stage_fast(y, p, None, w.H / 3, w.h, orc.opts(method=3, ramp=w.ramp))
    assert np.all(st == 0)
    y, st, _ = m.stage_fast(y, p, None, w.H * 5 / 12, w.h, orc.opts(method=3))
    assert np.all(st == 0)
    return w, m, y, p


def test_adaptive_stage_converges_to_fine_fixed_steps(orc):
    """The stage's global error follows the controller's tolerance (about the size of
    the tolerance, and 100x smaller for a 100x smaller tolerance), against fixed
    substeps 256 times smaller than the workload's."""
    w, m, y, p = _relaxed_box_cells(orc)
    phi = mechgen.random_forcing(3, y.shape[0], w.mech.n, 1)
    Hs = w.H / 4
    ref, rst, _ = m.stage_fast(y, p, phi, Hs, w.h / 256, orc.opts(method=3))
    assert np.all(rst == 0)
    errs = []
    for tol in (1e-5, 1e-7):
        out, st, _ = m.stage_fast(y, p, phi, Hs, w.h, orc.opts(method=3, adaptive=1, ctrl_rtol=tol,
                                                               ctrl_atol_Y=tol * 1e-6, ctrl_atol_T=tol))
        assert np.all(st == 0)
        errs.append(np.max(np.abs(out - ref) / np.maximum(np.abs(ref), 1e-6)))
    assert errs[0] < 3e-5 and errs[1] < 3e-7, errs
    assert errs[1] < 0.05 * errs[0]


def test_adaptive_stage_adapts_per_cell(orc):
    """Each cell takes its own number of steps: quiet cells far fewer than the fixed
    scheme's fine-tolerance equivalent, stiff ones more."""
    w, m, y, p = _relaxed_box_cells(orc, n=16, seed=2)
    out, st, ss = m.stage_fast(y, p, None, w.H / 4, w.h,
                               orc.opts(method=3, adaptive=1, ctrl_rtol=1e-7, ctrl_atol_Y=1e-13, ctrl_atol_T=1e-7))
    assert np.all(st == 0)
    steps = ss[:, 0]
    assert steps.max() >= 3 * steps.min(), steps


def test_adaptive_first_step_exponent(orc):
    """A per-cell first step (uniform substep times 2^k): k = 0 is the default
    exactly; other first steps change the step sequence but not the accuracy the
    controller delivers against the fine fixed-step solution."""
    w, m, y, p = _relaxed_box_cells(orc, n=8, seed=3)
    phi = mechgen.random_forcing(4, y.shape[0], w.mech.n, 1)
    Hs = w.H / 4
    tol = 1e-7
    o = orc.opts(method=3, adaptive=1, ctrl_rtol=tol, ctrl_atol_Y=tol * 1e-6, ctrl_atol_T=tol)
    base, st0, ss0 = m.stage_fast(y, p, phi, Hs, w.h, o)
    same, st1, ss1 = m.stage_fast(y, p, phi, Hs, w.h, o, step_exp=np.zeros(y.shape[0], np.int8))
    np.testing.assert_array_equal(same, base)
    np.testing.assert_array_equal(ss1, ss0)
    ref, rst, _ = m.stage_fast(y, p, phi, Hs, w.h / 256, orc.opts(method=3))
    assert np.all(rst == 0)
    k = np.array([-6, -3, -1, 1, 2, 3, -2, 0], np.int8)
    out, st, ss = m.stage_fast(y, p, phi, Hs, w.h, o, step_exp=k)
    assert np.all(st == 0)
    assert not np.array_equal(ss[:, 1], ss0[:, 1])          # other step sequences were taken
    err = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), 1e-6))
    assert err < 3e-7, err
