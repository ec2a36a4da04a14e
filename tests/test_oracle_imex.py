"""Pins of the oracle's implicit diffusion solve and first-order IMEX-MRI step:
the Fourier solve against the 7-point operator applied by finite differences, the
step reducing to backward Euler without chemistry and advection, and first-order
convergence to a fine single-rate solution of the coupled problem."""
import numpy as np
import pytest

import mechgen
from test_oracle_integrators import no_chemistry


def lap7(x, g):
    """D lap_h x by explicit neighbour differences (np.roll), [ncell][n] layout."""
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    X = x.reshape(nz, ny, nx, -1)
    out = np.zeros_like(X)
    for axis, N in ((2, nx), (1, ny), (0, nz)):
        if N > 1:
            out += (np.roll(X, 1, axis) - 2 * X + np.roll(X, -1, axis)) / g["dx"] ** 2
    return (g["D"] * out).reshape(x.shape)


@pytest.mark.parametrize("shape", [(16, 1, 1), (8, 6, 5), (7, 1, 9)])
def test_fourier_solve_satisfies_the_stencil(orc, shape):
    nx, ny, nz = shape
    g = dict(nx=nx, ny=ny, nz=nz, dx=1e-4, u=(0.0, 0.0, 0.0), D=1e-5, order=2)
    rng = np.random.default_rng(nx * ny * nz)
    b = rng.standard_normal((nx * ny * nz, 5))
    a = 3e-3                                # a D / dx^2 = 3: a stiff implicit stage
    x = orc.diffusion_solve(b, g, a)
    np.testing.assert_allclose(x - a * lap7(x, g), b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_imex1_without_chemistry_and_advection_is_backward_euler(orc):
    mech = no_chemistry()
    m = orc.Mech(mech)
    g = dict(nx=12, ny=1, nz=1, dx=1e-4, u=(0.0, 0.0, 0.0), D=1e-5, order=2)
    rng = np.random.default_rng(4)
    y = np.concatenate([rng.dirichlet(np.ones(3), 12), rng.uniform(500, 2000, (12, 1))], 1)
    H = 1e-3
    out, st, _ = orc.imex1_step(m, y, np.full(12, 101325.0), g, H, H / 10, orc.opts(method=3))
    assert np.all(st == 0)
    be = orc.diffusion_solve(y, g, H)
    np.testing.assert_allclose(out, be, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out - H * lap7(out, g), y, rtol=1e-11, atol=1e-14)


def test_imex1_converges_at_first_order(orc):
    """Coupled chemistry, advection and diffusion on a 1-D line against a fine
    single-rate SDIRK3 solution of the same semi-discrete system (2nd-order
    stencils): the error halves with H."""
    w = mechgen.workload("line64", cells_per_side=16)
    m = orc.Mech(w.mech)
    g = dict(w.grid, order=2, D=4e-4)          # diffusion stiff enough to want an implicit treatment
    t_end = 2e-8
    o = orc.opts(method=3, ramp=10)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, 1e-8, 1e-10, o)      # start past the initial transient
    ref = m.single_rate(y0, w.p, g, t_end, 800, orc.opts(method=3))
    errs = []
    for nsteps in (4, 8, 16):
        H = t_end / nsteps
        y = y0.copy()
        for s in range(nsteps):
            y, st, _ = orc.imex1_step(m, y, w.p, g, H, H / 10, orc.opts(method=3))
            assert np.all(st == 0)
        errs.append(np.max(np.abs(y[:, -1] - ref[:, -1])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.8) and np.all(rates < 1.3), (errs, rates)


def test_imex1_without_diffusion_is_one_mis_stage(orc):
    """With D = 0 the implicit correction is the identity (up to the rounding of the
    Fourier round trip), so the step is the fast stage over [0, H] with the
    constant advection forcing f^E(y_n)."""
    w = mechgen.workload("line64", cells_per_side=16)
    m = orc.Mech(w.mech)
    g = dict(w.grid, D=0.0)
    H = w.H / 2
    out, st, _ = orc.imex1_step(m, w.y0, w.p, g, H, w.h, orc.opts(method=w.method))
    assert np.all(st == 0)
    fE = orc.slow_rhs(w.y0, g)
    ref, rst, _ = m.stage_fast(w.y0, w.p, fE[:, None, :], H, w.h, orc.opts(method=w.method))
    assert np.all(rst == 0)
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-18)


def test_imex2_without_chemistry_and_advection_is_two_crank_nicolson_half_steps(orc):
    """No chemistry, no advection: the MRI step is the identity and the step is
    (I - (H/4) L)^-1 (I + (H/4) L) applied twice, checked with the dense periodic
    Laplacian and a dense solve."""
    mech = no_chemistry()
    m = orc.Mech(mech)
    nx = 10
    g = dict(nx=nx, ny=1, nz=1, dx=1e-4, u=(0.0, 0.0, 0.0), D=1e-5, order=2)
    rng = np.random.default_rng(6)
    y = np.concatenate([rng.dirichlet(np.ones(3), nx), rng.uniform(500, 2000, (nx, 1))], 1)
    H = 2e-3
    out, st, _ = orc.imex2_step(m, y, np.full(nx, 101325.0), g, H, H / 10, orc.opts(method=3))
    assert np.all(st == 0)
    Ld = (np.roll(np.eye(nx), 1, 1) + np.roll(np.eye(nx), -1, 1) - 2 * np.eye(nx)) * g["D"] / g["dx"] ** 2
    a = H / 4
    S = np.linalg.solve(np.eye(nx) - a * Ld, np.eye(nx) + a * Ld)
    np.testing.assert_allclose(out, S @ (S @ y), rtol=1e-12, atol=1e-15)


def test_imex2_converges_at_second_order(orc):
    """The coupled line problem of the first-order test: the Strang-split step's
    error falls by about four when H halves."""
    w = mechgen.workload("line64", cells_per_side=16)
    m = orc.Mech(w.mech)
    g = dict(w.grid, order=2, D=4e-4)
    t_end = 2e-8
    o = orc.opts(method=3, ramp=10)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, 1e-8, 1e-10, o)      # start past the initial transient
    g2 = dict(g, order=2)
    ref = m.single_rate(y0, w.p, g2, t_end, 800, orc.opts(method=3))
    errs = []
    for nsteps in (4, 8, 16):
        H = t_end / nsteps
        y = y0.copy()
        for s in range(nsteps):
            y, st, _ = orc.imex2_step(m, y, w.p, g, H, H / 10, orc.opts(method=3))
            assert np.all(st == 0)
        errs.append(np.max(np.abs(y[:, -1] - ref[:, -1])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print("errors", errs, "rates", rates)
    assert np.all(rates > 1.7) and np.all(rates < 2.5), (errs, rates)


def test_imex2_without_diffusion_is_one_mri3_step(orc):
    """With D = 0 both Crank-Nicolson half steps are the identity (up to the rounding
    of the Fourier round trips), so the step is the MRI3 step with the advection."""
    w = mechgen.workload("line64", cells_per_side=16)
    m = orc.Mech(w.mech)
    g = dict(w.grid, D=0.0)
    out, st, _ = orc.imex2_step(m, w.y0, w.p, g, w.H, w.h, orc.opts(method=w.method, ramp=w.ramp))
    assert np.all(st == 0)
    ref, rst, _ = m.mri_step(w.y0, w.p, g, w.H, w.h, orc.opts(method=w.method, ramp=w.ramp))
    assert np.all(rst == 0)
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-18)
