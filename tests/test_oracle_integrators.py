"""Pins of the oracle's time integration: SDIRK order conditions and observed
order, the KW3 slow method's order conditions, reductions of the MRI stage and
step to plain quadrature / plain ERK3 / plain sub-cycling, the multirate KPR
convergence order, conservation by the fast solve, and a brute-force coupled
single-rate reference on a few cells."""
import numpy as np
import pytest

import mechgen

R_U = 8.314462618


# --------------------------------------------------------------------------- tableaux

@pytest.mark.parametrize("method", [2, 3])
def test_sdirk_order_conditions_and_L_stability(orc, method):
    A, b, c = orc.sdirk_tableau(method)
    s = len(b)
    g = A[0, 0]
    assert np.allclose(np.diag(A), g, rtol=0, atol=1e-15)          # singly diagonal
    assert np.allclose(np.triu(A, 1), 0.0)                          # diagonally implicit
    np.testing.assert_allclose(A.sum(1), c, atol=1e-15)             # row sums
    np.testing.assert_allclose(b, A[-1], atol=0)                    # stiffly accurate
    assert b.sum() == pytest.approx(1.0, abs=1e-15)
    assert b @ c == pytest.approx(0.5, abs=1e-15)
    if method == 3:
        assert b @ c ** 2 == pytest.approx(1.0 / 3.0, abs=1e-15)
        assert b @ A @ c == pytest.approx(1.0 / 6.0, abs=1e-15)
        assert g ** 3 - 3 * g ** 2 + 1.5 * g - 1.0 / 6.0 == pytest.approx(0.0, abs=1e-15)
        assert 0.43 < g < 0.44
    else:
        assert g == pytest.approx(1.0 - 1.0 / np.sqrt(2.0), abs=1e-16)
    # stability function R(z) = 1 + z b^T (I - z A)^{-1} 1 -> 0 as z -> -inf (L-stability)
    for z in (-1e6, -1e10):
        R = 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
        assert abs(R) < 1e-5
    # A-stability sample on the imaginary axis
    for w in (0.1, 1.0, 10.0, 100.0):
        z = 1j * w
        R = 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
        assert abs(R) <= 1.0 + 1e-12


def test_kw3_order_conditions_and_coupling(orc):
    A, c = orc.mri_tableau()
    b = A[3, :3]
    Ae = A[:3, :3]
    ce = c[:3]
    np.testing.assert_allclose(A.sum(1), c, atol=1e-15)
    assert b.sum() == pytest.approx(1.0, abs=1e-15)
    assert b @ ce == pytest.approx(0.5, abs=1e-15)
    assert b @ ce ** 2 == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert b @ Ae @ ce == pytest.approx(1.0 / 6.0, abs=1e-15)
    G = orc.mri_coupling()
    # each stage's constant forcing is a consistent average of slow evaluations
    np.testing.assert_allclose(G[1:].sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(G[1, :1], [1.0], atol=1e-15)
    np.testing.assert_allclose(G[2, :2], [-5.0 / 4.0, 9.0 / 4.0], atol=1e-14)
    np.testing.assert_allclose(G[3, :3], [17.0 / 12.0, -51.0 / 20.0, 32.0 / 15.0], atol=1e-14)


@pytest.mark.parametrize("method,order", [(2, 2), (3, 3)])
def test_sdirk_observed_order_linear(orc, method, order):
    errs = []
    for N in (10, 20, 40, 80):
        y = orc.sdirk_scalar(method, 0, -1.0, 0.0, 1.0, N, 1.0)
        errs.append(abs(y - np.exp(-1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(rates[-1] - order) < 0.1, rates


@pytest.mark.parametrize("method", [2, 3])
def test_sdirk_prothero_robinson_stiff(orc, method):
    """y' = lam (y - cos t) - sin t, y(0) = 1, exact cos t; for lam = -1e8 the
    stiffly accurate L-stable methods track the smooth solution with errors far
    below h (no order reduction to zero, no instability)."""
    for N in (10, 40):
        y = orc.sdirk_scalar(method, 1, -1e8, 0.0, 1.0, N, 1.0)
        assert abs(y - np.cos(1.0)) < 1e-6


# --------------------------------------------------------------------------- stage reductions

def no_chemistry(Ns=3):
    """A mechanism with no reactions: f^F == 0."""
    nasa = np.zeros((Ns, 7))
    nasa[:, 0] = 3.5
    return mechgen.Mechanism(["H"], np.ones((Ns, 1), np.int32), np.linspace(0.002, 0.03, Ns), nasa,
                             np.zeros(0, np.int32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32),
                             np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0), np.zeros(0),
                             np.zeros((0, Ns)), np.zeros((0, 7)))


@pytest.mark.parametrize("method,K", [(2, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
@pytest.mark.parametrize("ramp", [0, 5])
def test_stage_without_chemistry_is_exact_quadrature(orc, method, K, ramp):
    """f^F == 0: the stage integrates the polynomial forcing exactly,
    v(T_i) = y + Hs sum_k phi_k / (k + 1), for degrees the method's quadrature
    (order conditions b.c^k = 1/(k+1)) integrates exactly."""
    mech = no_chemistry()
    m = orc.Mech(mech)
    rng = np.random.default_rng(K)
    ncell = 5
    y = np.concatenate([rng.dirichlet(np.ones(3), ncell), rng.uniform(500, 2000, (ncell, 1))], 1)
    phi = rng.standard_normal((ncell, K, 4)) * np.array([1e3, 1e3, 1e3, 1e7])
    Hs, h = 3e-8, 1e-9
    out, st, stats = m.stage_fast(y, np.full(ncell, 101325.0), phi, Hs, h, orc.opts(method=method, ramp=ramp))
    assert np.all(st == 0)
    expect = y + Hs * sum(phi[:, k, :] / (k + 1) for k in range(K))
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-16)
    assert np.all(stats[:, 0] == 30 + ramp)


def test_stage_substep_count(orc):
    """n_i = ceil(Hs/h) uniform substeps; the ramp replaces the first by ramp+1."""
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    H = w.H
    for dc, expect in ((1 / 3, 34), (5 / 12, 42), (1 / 4, 25)):
        _, _, stats = m.stage_fast(w.y0[:2], w.p[:2], None, dc * H, w.h, orc.opts(method=2))
        assert np.all(stats[:, 0] == expect)


# --------------------------------------------------------------------------- MRI step reductions

def test_mri_without_chemistry_is_erk3(orc):
    """f^F == 0: the MIS-form MRI step is exactly the Knoth-Wolke ERK3 step on f^S."""
    mech = no_chemistry()
    m = orc.Mech(mech)
    g = dict(nx=12, ny=1, nz=1, dx=1e-4, u=(1.0, 0.0, 0.0), D=1e-5, order=2)
    rng = np.random.default_rng(3)
    x = np.arange(12) / 12
    y = np.stack([0.3 + 0.1 * np.sin(2 * np.pi * x), 0.3 + 0.1 * np.cos(2 * np.pi * x), np.full(12, 0.4),
                  1000 + 300 * np.sin(4 * np.pi * x)], 1) + rng.uniform(0, 1e-3, (12, 4))
    H = 1e-6
    out, st, _ = m.mri_step(y, np.full(12, 101325.0), g, H, H / 10, orc.opts(method=3))
    f = lambda v: orc.slow_rhs(v, g)
    k1 = f(y)
    k2 = f(y + H * (1 / 3) * k1)
    k3 = f(y + H * (-3 / 16 * k1 + 15 / 16 * k2))
    expect = y + H * (1 / 6 * k1 + 3 / 10 * k2 + 8 / 15 * k3)
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-15)


def test_mri_without_transport_is_subcycled_chemistry(orc):
    """f^S == 0 (u = D = 0): the forcing vanishes and the step is the plain fast
    integration over the three stage intervals (Lie-Trotter structure with r = 0)."""
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    g = dict(w.grid, u=(0.0, 0.0, 0.0), D=0.0)
    o = orc.opts(method=2)
    out, st, _ = m.mri_step(w.y0, w.p, g, w.H, w.h, o)
    y = w.y0
    for dc in (1 / 3, 5 / 12, 1 / 4):
        y, _, _ = m.stage_fast(y, w.p, None, dc * w.H, w.h, o)
    np.testing.assert_array_equal(out, y)


def test_slow_rhs_exact_on_polynomials(orc):
    """Central differences are exact for low-degree polynomials: on a periodic
    grid use a single Fourier mode and compare with the stencil's symbol."""
    for order in (2, 4):
        nx, dx = 32, 1e-3
        x = np.arange(nx) * dx
        L = nx * dx
        kw = 2 * np.pi / L
        y = np.stack([np.sin(kw * x), np.cos(kw * x)], 1)
        g = dict(nx=nx, ny=1, nz=1, dx=dx, u=(2.0, 0, 0), D=3e-4, order=order)
        f = orc.slow_rhs(y, g)
        th = kw * dx
        if order == 2:
            d1, d2 = np.sin(th) / dx, -(2 - 2 * np.cos(th)) / dx ** 2
        else:
            d1 = (8 * np.sin(th) - np.sin(2 * th)) / (6 * dx)
            d2 = -(30 - 32 * np.cos(th) + 2 * np.cos(2 * th)) / (12 * dx ** 2)
        # d/dx sin -> d1 cos, d2/dx2 sin -> d2 sin (discrete symbols)
        expect0 = -2.0 * d1 * np.cos(kw * x) + 3e-4 * d2 * np.sin(kw * x)
        expect1 = 2.0 * d1 * np.sin(kw * x) + 3e-4 * d2 * np.cos(kw * x)
        np.testing.assert_allclose(f[:, 0], expect0, atol=1e-9 * np.abs(expect0).max())
        np.testing.assert_allclose(f[:, 1], expect1, atol=1e-9 * np.abs(expect1).max())


# --------------------------------------------------------------------------- KPR convergence

@pytest.mark.parametrize("fast,lo,hi", [(3, 2.8, 3.3), (2, 1.8, 2.3)])
def test_kpr_multirate_convergence_order(orc, fast, lo, hi):
    """Multirate KPR problem with closed-form solution.  KW3 slow + SDIRK3 fast at
    fixed H/h converges at order 3; with SDIRK2 fast the order drops to 2, as the
    paper observes for its second-order fast method (Sec. 5.2)."""
    errs = []
    steps = (20, 40, 80, 160) if fast == 3 else (40, 80, 160, 320)
    for N in steps:
        e, _ = orc.kpr_mri(fast, -1.0, 0.5, 1.0, 20.0, 1.0, N, 5)
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert lo <= rates[-1] <= hi, (errs, rates)


def test_kpr_rhs_vanishes_at_exact_solution():
    """Self-check of the KPR construction: Phi = 0 on the exact solution, so the
    right-hand side equals the exact derivative."""
    beta, omega, G, e = 1.0, 20.0, -1.0, 0.5
    for t in np.linspace(0, 3, 7):
        u = np.sqrt(3 + np.cos(beta * t))
        v = np.sqrt(2 + np.cos(omega * t))
        pu = (-3 + u * u - np.cos(beta * t)) / (2 * u)
        pv = (-2 + v * v - np.cos(omega * t)) / (2 * v)
        assert abs(pu) < 1e-15 and abs(pv) < 1e-15
        du = G * pu + e * pv - beta * np.sin(beta * t) / (2 * u)
        assert du == pytest.approx(-beta * np.sin(beta * t) / (2 * u), abs=1e-15)


# --------------------------------------------------------------------------- conservation

def test_fast_solve_conserves_mass_and_elements(orc):
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    out, st, _ = m.stage_fast(w.y0, w.p, None, w.H, w.h, orc.opts(method=2, ramp=8))
    assert np.all(st == 0)
    np.testing.assert_allclose(out[:, :-1].sum(1), w.y0[:, :-1].sum(1), rtol=0, atol=1e-13)
    E = w.mech.elem / w.mech.W[:, None]
    np.testing.assert_allclose(out[:, :-1] @ E, w.y0[:, :-1] @ E, rtol=1e-12)


def test_mri_step_conserves_mass_and_elements(orc):
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    out, st, _ = m.mri_step(w.y0, w.p, w.grid, w.H, w.h, orc.opts(method=2, ramp=8))
    assert np.all(st == 0)
    np.testing.assert_allclose(out[:, :-1].sum(1), 1.0, rtol=0, atol=1e-13)
    E = w.mech.elem / w.mech.W[:, None]
    # the periodic transport only moves element mass around: grid totals are conserved
    np.testing.assert_allclose((out[:, :-1] @ E).sum(0), (w.y0[:, :-1] @ E).sum(0), rtol=1e-12)


# --------------------------------------------------------------------------- brute force

def test_mri_matches_brute_force_single_rate(orc):
    """Four coupled cells: the MRI step (KW3 + SDIRK3) against a single-rate SDIRK3
    integration of the full f^F + f^S with 1000x smaller steps.  The MRI error must be
    within 10x its own Richardson estimate |MRI(H) - MRI(H/2)| * 8/7."""
    w = mechgen.workload("line64", cells_per_side=4)
    m = orc.Mech(w.mech)
    g = dict(w.grid, u=(20.0, 0.0, 0.0), D=2e-4)
    o = orc.opts(method=3, rtol=1e-12, max_newton=40, ramp=10)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, 2e-9, 2e-9, o)    # move onto the fast manifold first
    H = 2e-8
    one, st, _ = m.mri_step(y0, w.p, g, H, H / 8, orc.opts(method=3, rtol=1e-12, max_newton=40))
    assert np.all(st == 0)
    half = y0
    for _ in range(2):
        half, st, _ = m.mri_step(half, w.p, g, H / 2, H / 16, orc.opts(method=3, rtol=1e-12, max_newton=40))
    ref = m.single_rate(y0, w.p, g, H, 800, orc.opts(method=3, rtol=1e-12, max_newton=40))
    scale = np.abs(ref).max(0)
    err = np.abs(one - ref).max(0) / scale
    est = np.abs(one - half).max(0) / scale * 8 / 7
    assert np.all(err <= 10 * est + 1e-13), (err, est)
    assert err.max() < 1e-4


def test_mri3_slow_evaluations_match_table2(orc):
    """Table 2 counts 97 slow evaluations for the third-order MRI method over 32 steps:
    one per stage start (the columns of the coupling matrix in use) per step, plus
    the initial evaluation (tests/golden/table2_mri3_slow_evals.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_mri3_slow_evals.txt")
    rec = dict(line.split() for line in open(path) if line.strip() and not line.startswith("#"))
    G = orc.mri_coupling()
    per_step = int(np.count_nonzero(np.any(G != 0.0, axis=0)))
    assert per_step == 3
    assert per_step * int(rec["steps"]) + 1 == int(rec["slow_evals"])
