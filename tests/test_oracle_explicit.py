"""Pins of the oracle's explicit fast integrators (the paper's MRI-P(k) fast methods,
Sec. 3.2): Heun's second-order method (code 12), Kutta's third-order method (13) and
the classical fourth-order Runge-Kutta method (14).  Their tableaux satisfy the
order conditions, their stability function is the truncated exponential series, one
step on y' = lambda y reproduces it, they converge at their orders on scalar
problems, integrate polynomial forcing exactly up to their quadrature order, set the
multirate order of the MRI step on the KPR problem, and on relaxed chemistry agree
with the (separately pinned) SDIRK3 solution as the substep shrinks."""
import math

import numpy as np
import pytest

import mechgen
from test_oracle_integrators import no_chemistry

ORDER = {12: 2, 13: 3, 14: 4}


@pytest.mark.parametrize("method", [12, 13, 14])
def test_erk_order_conditions(orc, method):
    A, b, c = orc.erk_tableau(method)
    p = ORDER[method]
    assert len(b) == p                                   # s = p stages (p <= 4)
    assert np.all(np.triu(A) == 0.0)                     # explicit
    np.testing.assert_allclose(A.sum(1), c, atol=1e-16)  # row sums
    assert b.sum() == pytest.approx(1.0, abs=4e-16)
    assert b @ c == pytest.approx(1 / 2, abs=4e-16)
    if p >= 3:
        assert b @ c ** 2 == pytest.approx(1 / 3, abs=4e-16)
        assert b @ A @ c == pytest.approx(1 / 6, abs=4e-16)
    if p >= 4:
        assert b @ c ** 3 == pytest.approx(1 / 4, abs=4e-16)
        assert b @ (c * (A @ c)) == pytest.approx(1 / 8, abs=4e-16)
        assert b @ A @ c ** 2 == pytest.approx(1 / 12, abs=4e-16)
        assert b @ A @ A @ c == pytest.approx(1 / 24, abs=4e-16)
    # a condition of order p + 1 fails (the order is exactly p)
    fails = {2: b @ c ** 2 - 1 / 3, 3: b @ A @ A @ c - 1 / 24, 4: b @ c ** 4 - 1 / 5}[p]
    assert abs(fails) > 1e-3


@pytest.mark.parametrize("method", [12, 13, 14])
def test_erk_stability_function_is_truncated_exponential(orc, method):
    """R(z) = 1 + z b^T (I - z A)^-1 1 = sum_{k <= p} z^k / k! for s = p <= 4, and one
    step of the oracle on y' = lambda y multiplies y by R(h lambda)."""
    A, b, c = orc.erk_tableau(method)
    p = ORDER[method]
    for z in (-0.3, -1.7, 0.9, -2.5):
        R = 1.0 + z * b @ np.linalg.solve(np.eye(p) - z * A, np.ones(p))
        assert R == pytest.approx(sum(z ** k / math.factorial(k) for k in range(p + 1)), rel=1e-14)
        y1 = orc.erk_scalar(method, 0, z, 0.0, 1.0, 1, 1.0)
        assert y1 == pytest.approx(R, rel=1e-14)


@pytest.mark.parametrize("method", [12, 13, 14])
def test_erk_observed_order(orc, method):
    """y' = -y (exact e^{-t}) and Prothero-Robinson y' = lambda (y - cos t) - sin t with
    lambda = -5 (exact cos t): errors fall at the method's order as h halves."""
    p = ORDER[method]
    for problem, lam, exact, y0 in ((0, -1.0, math.exp(-1.0), 1.0), (1, -5.0, math.cos(1.0), 1.0)):
        errs = [abs(orc.erk_scalar(method, problem, lam, 0.0, 1.0, N, y0) - exact) for N in (20, 40, 80, 160)]
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert p - 0.2 <= rates[-1] <= p + 0.3, (method, problem, errs, rates)


@pytest.mark.parametrize("method,K", [(12, 1), (12, 2), (13, 1), (13, 3), (14, 2), (14, 4)])
@pytest.mark.parametrize("ramp", [0, 4])
def test_erk_stage_without_chemistry_is_exact_quadrature(orc, method, K, ramp):
    """f^F == 0: the stage integrates the polynomial forcing r = sum_k rhohat^k phi_k exactly,
    v(T_i) = y + Hs sum_k phi_k / (k + 1), up to degree K - 1 <= the quadrature order - 1
    (trapezoid rule for Heun, Simpson's rule for Kutta 3 and RK4)."""
    m = orc.Mech(no_chemistry())
    rng = np.random.default_rng(K + method)
    ncell = 5
    y = np.concatenate([rng.dirichlet(np.ones(3), ncell), rng.uniform(500, 2000, (ncell, 1))], 1)
    phi = rng.standard_normal((ncell, K, 4)) * np.array([1e3, 1e3, 1e3, 1e7])
    Hs, h = 3e-8, 1e-9
    out, st, stats = m.stage_fast(y, np.full(ncell, 101325.0), phi, Hs, h, orc.opts(method=method, ramp=ramp))
    assert np.all(st == 0)
    expect = y + Hs * sum(phi[:, k, :] / (k + 1) for k in range(K))
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-16)
    assert np.all(stats[:, 0] == 30 + ramp)
    assert np.all(stats[:, 1] == (30 + ramp) * ORDER[method])     # right-hand-side evaluations
    assert np.all(stats[:, 2] == 0)                                # no Jacobian


@pytest.mark.parametrize("fast,lo,hi", [(12, 1.8, 2.3), (13, 2.8, 3.3), (14, 2.8, 3.3)])
def test_kpr_multirate_order_with_explicit_fast_methods(orc, fast, lo, hi):
    """KW3 slow with an explicit fast method at fixed H/h: the multirate order is
    min(3, p) -- 2 with Heun, 3 with Kutta 3 and with RK4 (the slow method's order)."""
    errs = []
    # Heun's error constant reaches its asymptotic regime later (rates 2.3, 2.1, 1.7, 1.9, 1.95)
    for N in ((160, 320, 640, 1280) if fast == 12 else (20, 40, 80, 160)):
        e, _ = orc.kpr_mri(fast, -1.0, 0.5, 1.0, 20.0, 1.0, N, 5)
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert lo <= rates[-1] <= hi, (errs, rates)


@pytest.mark.parametrize("method", [12, 13, 14])
def test_erk_chemistry_converges_to_the_sdirk3_solution(orc, method):
    """On relaxed cells of the 9-species line over a stage of 4e-6 s, explicit substeps
    converge to the SDIRK3 solution of the same stage (16384 substeps): the difference
    falls at the method's order (a factor near 2^p) as the substep halves."""
    w = mechgen.workload("line64")
    m = orc.Mech(w.mech)
    idx = np.arange(0, 64, 8)
    y, st, _ = m.stage_fast(w.y0[idx], w.p[idx], None, w.H, w.h, orc.opts(method=3, ramp=w.ramp))
    assert np.all(st == 0)
    phi = mechgen.random_forcing(4, len(idx), w.mech.n, 1)
    Hs = 4e-6
    ref, st, _ = m.stage_fast(y, w.p[idx], phi, Hs, Hs / 16384, orc.opts(method=3, rtol=1e-13))
    assert np.all(st == 0)
    diffs = []
    for nsub in (16, 32, 64):
        out, st, _ = m.stage_fast(y, w.p[idx], phi, Hs, Hs / nsub, orc.opts(method=method))
        assert np.all(st == 0)
        scale = np.maximum(np.abs(ref), 1e-10)
        diffs.append(float(np.max(np.abs(out - ref) / scale)))
    p = ORDER[method]
    ratios = np.array(diffs[:-1]) / np.array(diffs[1:])
    assert np.all((ratios > 0.75 * 2 ** p) & (ratios < 1.4 * 2 ** p)), (diffs, ratios)
    assert diffs[-1] < 1e-4
