"""Pins of the oracle's rate magnitudes: the Lindemann-Troe falloff blending, the
third-body concentration [M], the temperature exponent of the Arrhenius law and
the energy row of the fast right-hand side.

None of these can be pinned by detailed balance (it fixes k_f / k_r, not k_f),
by conservation of mass and elements (which say nothing about T) or by the
complex-step Jacobian (which differentiates whatever the RHS computes).  The
pins here rest on properties that hold whatever the implementation:

* Arrhenius (Sec. 3: the kinetics the paper names, in the standard Chemkin
  form k = A T^b exp(-Ta/T)): ratios k(T1)/k(T2) at Ta = 0 are (T1/T2)^b, at
  b = 0 they are exp(-Ta (1/T1 - 1/T2));
* Lindemann falloff: k/k_inf -> 1 as P_r -> infinity, k/(k_0 [M]) -> 1 as
  P_r -> 0, k = k_inf / 2 at P_r = 1 (k_inf and k_0 read from plain reactions
  with the same Arrhenius parameters);
* Troe broadening (Gilbert, Luther & Troe 1983; c = -0.4 - 0.67 log F_cent,
  n' = 0.75 - 1.27 log F_cent, d = 0.14, log = log10): F = F_cent exactly where
  log P_r + c = 0, F = sqrt(F_cent) where log P_r + c = n'/(1 + d) or
  -n'/(1 - d), and F = 1 where log P_r + c = n'/d (the pole of the broadening
  argument).  F_cent is made a single known number by sending the other terms'
  temperatures to their limits;
* third body: with the products absent, q scales as lambda^(order + 1) when
  every concentration scales by lambda; moving concentration between two inert
  collision partners changes q in proportion to sum_k alpha_k C_k;
* energy: a constant-pressure adiabatic cell keeps its specific enthalpy,
  so sum_k h_k f_{Y_k} + cp f_T = 0 at every state (h_k, cp per unit mass), and
  a fast stage without forcing keeps h(Y, T) up to the integrator's own error,
  which falls at the method's order as the substep shrinks.
"""
import numpy as np
import pytest

import mechgen

R_U = 8.314462618
P_ATM = 101325.0
TROE_D = 0.14


def _nasa_const(Ns, a6=None, a7=None):
    nasa = np.zeros((Ns, 7))
    nasa[:, 0] = 3.5
    nasa[:, 5] = a6 if a6 is not None else np.linspace(-800.0, 600.0, Ns)
    nasa[:, 6] = a7 if a7 is not None else np.linspace(2.0, 6.0, Ns)
    return nasa


def _mech(rtype, reac, prod, A, b, Ta, eff_rows=(), troe_rows=(), eff_row=None, troe_row=None, Ns=5,
          W=None):
    """A hand-built mechanism over species 0..Ns-1 (one element; the element counts are
    not used by the rates)."""
    R = len(rtype)
    r = -np.ones((R, 3), np.int32)
    p = -np.ones((R, 3), np.int32)
    for i in range(R):
        r[i, :len(reac[i])] = reac[i]
        p[i, :len(prod[i])] = prod[i]
    W = np.array(W if W is not None else [0.002, 0.016, 0.018, 0.028, 0.032][:Ns], float)
    return mechgen.Mechanism(
        ["H"], np.ones((Ns, 1), np.int32), W, _nasa_const(Ns), np.array(rtype, np.int32), r, p,
        np.array(eff_row if eff_row is not None else [-1] * R, np.int32),
        np.array(troe_row if troe_row is not None else [-1] * R, np.int32),
        np.array(A, float), np.array(b, float), np.array(Ta, float),
        np.array(eff_rows, float).reshape(len(eff_rows), Ns), np.array(troe_rows, float).reshape(len(troe_rows), 7))


# ------------------------------------------------------------------------------ Arrhenius

@pytest.mark.parametrize("b", [-1.3, -0.4, 0.7, 1.5])
def test_arrhenius_temperature_exponent(orc, b):
    """Ta = 0: k(2T)/k(T) = 2^b and k(3T)/k(T) = 3^b; b enters as a power of T."""
    m = orc.Mech(_mech([0], [[0, 1]], [[2]], [3.0e-4], [b], [0.0]))
    C = np.ones(5)
    for T in (350.0, 800.0, 1000.0):
        k1 = m.rate_coeffs(T, C)[0][0]
        k2 = m.rate_coeffs(2 * T, C)[0][0]
        k3 = m.rate_coeffs(3 * T, C)[0][0]
        assert k2 / k1 == pytest.approx(2.0 ** b, rel=1e-13)
        assert k3 / k1 == pytest.approx(3.0 ** b, rel=1e-13)


def test_arrhenius_activation_temperature(orc):
    """b = 0: k(T1)/k(T2) = exp(-Ta (1/T1 - 1/T2)); with both, the product of the two."""
    Ta, b = 9000.0, 0.8
    m = orc.Mech(_mech([0, 0], [[0, 1], [0, 1]], [[2], [2]], [2.0, 2.0], [0.0, b], [Ta, Ta]))
    C = np.ones(5)
    T1, T2 = 700.0, 1900.0
    k1, k2 = m.rate_coeffs(T1, C)[0], m.rate_coeffs(T2, C)[0]
    assert k1[0] / k2[0] == pytest.approx(np.exp(-Ta * (1 / T1 - 1 / T2)), rel=1e-12)
    assert k1[1] / k2[1] == pytest.approx((T1 / T2) ** b * np.exp(-Ta * (1 / T1 - 1 / T2)), rel=1e-12)
    # the pre-exponential factor multiplies: k = A at T = 1 K with b = 0, Ta = 0
    m1 = orc.Mech(_mech([0], [[0, 1]], [[2]], [7.5], [0.0], [0.0]))
    assert m1.rate_coeffs(1234.0, C)[0][0] == pytest.approx(7.5, rel=1e-15)


# ------------------------------------------------------------------------------ falloff

# species: 0 A, 1 B, 2 AB, 3 X (inert partner), 4 Z (inert partner)
K_INF = (4.0e5, 0.6, 3000.0)      # A, b, Ta of the high-pressure limit
K_0 = (9.0e7, -1.1, 800.0)        # A0, b0, Ta0 of the low-pressure limit


def _falloff_mech(a, T3, T1, T2, eff=(1.0, 1.0, 1.0, 2.5, 0.4)):
    """Reaction 0: A + B (+M) <=> AB, Lindemann/Troe with (a, T***, T*, T**); reaction 1: a
    plain reaction with the high-pressure Arrhenius parameters (k_inf); reaction 2: a
    plain reaction with the low-pressure ones (k_0)."""
    return _mech([2, 0, 0], [[0, 1], [0, 1], [0, 1]], [[2], [2], [2]],
                 [K_INF[0], K_INF[0], K_0[0]], [K_INF[1], K_INF[1], K_0[1]], [K_INF[2], K_INF[2], K_0[2]],
                 eff_rows=[eff], troe_rows=[[K_0[0], K_0[1], K_0[2], a, T3, T1, T2]],
                 eff_row=[0, -1, -1], troe_row=[0, -1, -1])


def _partners_for_M(M, eff=(1.0, 1.0, 1.0, 2.5, 0.4)):
    """Concentrations with [M] = sum alpha_k C_k = M, most of it from the inert partner X."""
    C = np.array([1e-3, 2e-3, 5e-4, 0.0, 0.0]) * M
    C[4] = 0.1 * M
    rest = M - float(np.dot(eff, C))
    C[3] = rest / eff[3]
    assert C[3] > 0
    return C


def _k(m, T, C):
    kf = m.rate_coeffs(T, C)[0]
    return kf[0], kf[1], kf[2]      # falloff, k_inf, k_0


LINDEMANN = dict(a=0.0, T3=1e300, T1=1.0, T2=1e300)     # F_cent = e^{-T/T***} + e^{-T**/T} = 1


@pytest.mark.parametrize("T", [500.0, 1200.0, 2400.0])
def test_lindemann_limits_and_midpoint(orc, T):
    m = orc.Mech(_falloff_mech(**LINDEMANN))
    _, kinf, k0 = _k(m, T, np.ones(5))
    M1 = kinf / k0                                    # P_r = 1
    k, _, _ = _k(m, T, _partners_for_M(M1))
    assert k == pytest.approx(0.5 * kinf, rel=1e-13)
    k, _, _ = _k(m, T, _partners_for_M(1e9 * M1))     # high pressure
    assert k / kinf == pytest.approx(1.0, rel=2e-9)
    Mlo = 1e-9 * M1
    k, _, _ = _k(m, T, _partners_for_M(Mlo))          # low pressure: second order in [M]
    assert k / (k0 * Mlo) == pytest.approx(1.0, rel=2e-9)


def _troe_targets(Fc):
    lf = np.log10(Fc)
    c = -0.4 - 0.67 * lf
    nn = 0.75 - 1.27 * lf
    return c, nn


# F_cent reduced to one term by sending the others' temperatures to their limits
FCENT_CASES = [
    # a = 0, T** -> inf: F_cent = exp(-T/T***)
    (lambda T: dict(a=0.0, T3=T / np.log(1 / 0.45), T1=1.0, T2=1e300), 0.45),
    # a = 1, T** -> inf: F_cent = exp(-T/T*)
    (lambda T: dict(a=1.0, T3=1.0, T1=T / np.log(1 / 0.3), T2=1e300), 0.3),
    # a = 0.25, T*** -> 0, T* -> inf: F_cent = a + exp(-T**/T)
    (lambda T: dict(a=0.25, T3=1e-300, T1=1e300, T2=T * np.log(1 / 0.35)), 0.6),
]


@pytest.mark.parametrize("case", range(len(FCENT_CASES)))
@pytest.mark.parametrize("T", [600.0, 1800.0])
def test_troe_broadening_special_points(orc, case, T):
    par, Fc = FCENT_CASES[case]
    m = orc.Mech(_falloff_mech(**par(T)))
    _, kinf, k0 = _k(m, T, np.ones(5))
    c, nn = _troe_targets(Fc)
    # log10 Pr + c = 0: F = F_cent
    M = (kinf / k0) * 10.0 ** (-c)
    Pr = 10.0 ** (-c)
    k, _, _ = _k(m, T, _partners_for_M(M))
    assert k / (kinf * Pr / (1 + Pr)) == pytest.approx(Fc, rel=1e-12)
    # log10 Pr + c = n'/(1 + d): f1 = 1, F = sqrt(F_cent)
    u = nn / (1.0 + TROE_D)
    Pr = 10.0 ** (u - c)
    k, _, _ = _k(m, T, _partners_for_M((kinf / k0) * Pr))
    assert k / (kinf * Pr / (1 + Pr)) == pytest.approx(np.sqrt(Fc), rel=1e-12)
    # log10 Pr + c = -n'/(1 - d): f1 = -1, F = sqrt(F_cent) on the low-pressure side
    u = -nn / (1.0 - TROE_D)
    Pr = 10.0 ** (u - c)
    k, _, _ = _k(m, T, _partners_for_M((kinf / k0) * Pr))
    assert k / (kinf * Pr / (1 + Pr)) == pytest.approx(np.sqrt(Fc), rel=1e-12)
    # log10 Pr + c = n'/d: the denominator n' - d (log Pr + c) vanishes, f1 is unbounded
    # and F = 1 (no broadening)
    u = nn / TROE_D
    Pr = 10.0 ** (u - c)
    k, _, _ = _k(m, T, _partners_for_M((kinf / k0) * Pr))
    assert k / (kinf * Pr / (1 + Pr)) == pytest.approx(1.0, rel=1e-12)


def test_falloff_collision_efficiencies(orc):
    """[M] of a falloff reaction is efficiency-weighted: moving concentration from the
    inert partner X (alpha = 2.5) to Z (alpha = 0.4) moves P_r by the weighted sum (checked
    on the Lindemann form, where k = k_inf P_r/(1 + P_r))."""
    eff = (1.0, 1.0, 1.0, 2.5, 0.4)
    m = orc.Mech(_falloff_mech(**LINDEMANN))
    T = 1300.0
    _, kinf, k0 = _k(m, T, np.ones(5))
    C = _partners_for_M(kinf / k0)
    for delta in (0.1, 0.5, 0.9):
        C2 = C.copy()
        C2[4] += delta * C[3]
        C2[3] -= delta * C[3]
        Pr = k0 * float(np.dot(eff, C2)) / kinf
        k, _, _ = _k(m, T, C2)
        assert k == pytest.approx(kinf * Pr / (1 + Pr), rel=1e-13)


# ------------------------------------------------------------------------------ third body

def _thirdbody_mech(eff):
    # reaction 0: A + B + M <=> AB + M ; reaction 1 the same without M (plain)
    return _mech([1, 0], [[0, 1], [0, 1]], [[2], [2]], [5.0e2, 5.0e2], [0.3, 0.3], [1500.0, 1500.0],
                 eff_rows=[eff], eff_row=[0, -1])


def test_third_body_order_and_efficiencies(orc):
    eff = np.array([1.0, 1.0, 1.0, 2.5, 0.4])
    m = orc.Mech(_thirdbody_mech(eff))
    T = 1500.0
    C = np.array([3.0, 1.5, 0.0, 7.0, 4.0])          # products absent: q = k_f [M] C_A C_B
    q0 = m.progress(T, C)[0]
    for lam in (0.5, 2.0, 10.0):
        q = m.progress(T, lam * C)[0]
        assert q[0] / q0[0] == pytest.approx(lam ** 3, rel=1e-13)     # order 2 plus [M]
        assert q[1] / q0[1] == pytest.approx(lam ** 2, rel=1e-13)     # the plain twin
    # swapping inert partners moves q by the efficiency-weighted sum only
    M0 = float(np.dot(eff, C))
    for delta in (0.5, 3.0, 6.5):
        C2 = C.copy()
        C2[3] -= delta
        C2[4] += delta
        q = m.progress(T, C2)[0]
        assert q[0] / q0[0] == pytest.approx(float(np.dot(eff, C2)) / M0, rel=1e-13)
        assert q[1] == pytest.approx(q0[1], rel=1e-15)
    # and equals the plain twin's rate of progress times [M]
    assert q0[0] == pytest.approx(q0[1] * M0, rel=1e-13)


# ------------------------------------------------------------------------------ energy row

def _specific(m, mech, y):
    """Specific enthalpies h_k [J/kg] and mixture cp [J/(kg K)] from the oracle's NASA-7
    thermodynamics (pinned by the thermodynamic identities)."""
    T = y[-1]
    cpR, hRT, _, _ = m.thermo(T)
    h = hRT * R_U * T / mech.W
    cp = float(np.sum(y[:-1] * cpR * R_U / mech.W))
    return h, cp


@pytest.mark.parametrize("which", ["small", "medium"])
def test_energy_row_conserves_enthalpy(orc, which):
    """Adiabatic constant pressure: sum_k h_k dY_k/dt + cp dT/dt = 0 at every state."""
    spec = mechgen.MECH_SMALL if which == "small" else mechgen.MECH_MEDIUM
    mech = mechgen.make_mechanism(1000 if which == "small" else 3000, **spec)
    m = orc.Mech(mech)
    rng = np.random.default_rng(5)
    for _ in range(10):
        Y = rng.dirichlet(np.ones(mech.n_species))
        y = np.concatenate([Y, [rng.uniform(600, 2400)]])
        f = m.rhs(y, rng.uniform(0.5, 2.0) * P_ATM)
        h, cp = _specific(m, mech, y)
        gross = float(np.sum(np.abs(h * f[:-1])))
        assert gross > 0
        assert abs(float(np.dot(h, f[:-1])) + cp * f[-1]) <= 1e-12 * gross
        # the heat release has the sign of the enthalpy drop: T rises where sum h dY/dt < 0
        assert np.sign(f[-1]) == -np.sign(float(np.dot(h, f[:-1])))


def test_fast_stage_keeps_enthalpy(orc):
    """A fast stage without forcing keeps h(Y, T) = sum Y_k h_k(T) up to the SDIRK3
    discretisation error.  The stiff start-up transient is where the integrator loses
    the (nonlinear) invariant, so the drift is small against the heat release cp |dT|
    (a wrong sign or scale of f_T would make it of order one) and shrinks as the
    substeps resolve the transient."""
    import oracle
    mech = mechgen.make_mechanism(3000, **mechgen.MECH_MEDIUM)
    m = orc.Mech(mech)
    rng = np.random.default_rng(9)
    Y = rng.dirichlet(np.ones(mech.n_species), size=3)
    y0 = np.concatenate([Y, np.array([[1400.0], [1800.0], [2200.0]])], axis=1)
    p = np.full(3, P_ATM)
    Hs = 1e-8
    drifts = []
    for nsub in (16, 256):
        y, st, _ = m.stage_fast(y0, p, None, Hs, Hs / nsub, oracle.opts(method=3, rtol=1e-13, ramp=16), nthreads=3)
        assert np.all(st == 0)
        d = []
        for c in range(3):
            h0, cp0 = _specific(m, mech, y0[c])
            h1, _ = _specific(m, mech, y[c])
            dT = abs(y[c, -1] - y0[c, -1])
            assert dT > 10.0                     # the chemistry does move T
            d.append(abs(float(np.dot(y[c, :-1], h1)) - float(np.dot(y0[c, :-1], h0))) / (cp0 * dT))
        drifts.append(np.array(d))
    assert drifts[0].max() < 1e-4
    assert np.all(drifts[1] < drifts[0])
