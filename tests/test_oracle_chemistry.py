"""Pins of the oracle's thermodynamics, kinetics, Jacobian and LU against facts
that do not come from the oracle itself: thermodynamic identities, a closed-form
equilibrium constant, Gibbs-energy minimisation, conservation laws, complex-step
derivatives and LAPACK."""
import numpy as np
import pytest
import scipy.optimize

import mechgen

R_U = 8.314462618
P_ATM = 101325.0


def small():
    return mechgen.make_mechanism(1000, **mechgen.MECH_SMALL)


def medium():
    return mechgen.make_mechanism(3000, **mechgen.MECH_MEDIUM)


def random_states(mech, n, seed, Tlo=400.0, Thi=2400.0):
    rng = np.random.default_rng(seed)
    Y = rng.dirichlet(np.ones(mech.n_species), size=n)
    T = rng.uniform(Tlo, Thi, n)
    return np.concatenate([Y, T[:, None]], axis=1)


def one_reaction_mech(nasa, reac, prod, A=1.0, b=0.0, Ta=0.0, W=(0.002, 0.016, 0.018)):
    """A hand-built mechanism with one plain reversible reaction."""
    Ns = len(W)
    r = -np.ones((1, 3), np.int32)
    p = -np.ones((1, 3), np.int32)
    r[0, :len(reac)] = reac
    p[0, :len(prod)] = prod
    return mechgen.Mechanism(["H"], np.ones((Ns, 1), np.int32), np.array(W, float), np.array(nasa, float),
                             np.zeros(1, np.int32), r, p, -np.ones(1, np.int32), -np.ones(1, np.int32),
                             np.array([A]), np.array([b]), np.array([Ta]), np.zeros((0, Ns)), np.zeros((0, 7)))


# --------------------------------------------------------------------------- thermo

@pytest.mark.parametrize("mk", [small, medium])
def test_nasa_thermodynamic_identities(orc, mk):
    """dh/dT = cp and ds/dT = cp/T (h = RT h/RT, s = R s/R), g = h - Ts."""
    m = orc.Mech(mk())
    for T in (350.0, 900.0, 1700.0, 2600.0):
        cp, hRT, sR, gRT = m.thermo(T)
        d = 1e-3 * T
        hs = {}
        ss = {}
        for k in (-2, -1, 1, 2):
            _, hk, sk, _ = m.thermo(T + k * d)
            hs[k] = (T + k * d) * hk
            ss[k] = sk
        # five-point central differences, truncation O(d^4)
        dh = (-hs[2] + 8 * hs[1] - 8 * hs[-1] + hs[-2]) / (12 * d)
        ds = (-ss[2] + 8 * ss[1] - 8 * ss[-1] + ss[-2]) / (12 * d)
        np.testing.assert_allclose(dh, cp, rtol=1e-10)
        np.testing.assert_allclose(ds, cp / T, rtol=1e-10)
        np.testing.assert_allclose(gRT, hRT - sR, rtol=0, atol=1e-12 * np.abs(hRT).max())


def test_equilibrium_constant_closed_form(orc):
    """A <=> B + C with NASA polynomials reduced to constants: g/RT = a6/T - a7, so
    K_c = exp(-(sum nu a6)/T + sum nu a7) (p_atm / (R T))^(+1)."""
    nasa = np.zeros((3, 7))
    nasa[:, 5] = [-3000.0, 1000.0, 500.0]
    nasa[:, 6] = [1.0, -2.0, 0.5]
    mech = one_reaction_mech(nasa, [0], [1, 2], A=5.0, b=0.0, Ta=100.0)
    m = orc.Mech(mech)
    for T in (500.0, 1500.0):
        kf, kr, Kc = m.rate_coeffs(T, np.ones(3))
        expect = np.exp(-(1000.0 + 500.0 + 3000.0) / T + (-2.0 + 0.5 - 1.0)) * P_ATM / (R_U * T)
        assert Kc[0] == pytest.approx(expect, rel=1e-13)
        assert kf[0] == pytest.approx(5.0 * np.exp(-100.0 / T), rel=1e-14)
        assert kr[0] == pytest.approx(kf[0] / expect, rel=1e-13)


@pytest.mark.parametrize("mk", [small, medium])
def test_generated_kc_range(orc, mk):
    """The generator's promise: every K_c within 1e-30..1e30 on 300..3000 K."""
    mech = mk()
    m = orc.Mech(mech)
    for T in np.linspace(300, 3000, 64):
        _, _, Kc = m.rate_coeffs(T, np.ones(m.Ns))
        assert np.all(np.abs(np.log(Kc)) <= np.log(1e30))


# --------------------------------------------------------------------------- conservation

@pytest.mark.parametrize("mk", [small, medium])
def test_production_rates_conserve_mass_and_elements(orc, mk):
    mech = mk()
    m = orc.Mech(mech)
    # every reaction conserves elements
    for r in range(mech.n_reactions):
        ra = [i for i in mech.reac[r] if i >= 0]
        pa = [i for i in mech.prod[r] if i >= 0]
        np.testing.assert_array_equal(mech.elem[ra].sum(0), mech.elem[pa].sum(0))
    rng = np.random.default_rng(1)
    for _ in range(20):
        T = rng.uniform(400, 2500)
        C = rng.uniform(0.0, 10.0, m.Ns)
        q, w = m.progress(T, C)
        scale = np.abs(q).sum() * mech.W.max() + 1e-300
        assert abs(np.dot(mech.W, w)) <= 1e-13 * scale
        for e in range(mech.elem.shape[1]):
            sc = np.abs(q).sum() * mech.elem[:, e].max() + 1e-300
            assert abs(np.dot(mech.elem[:, e], w)) <= 1e-13 * sc


# --------------------------------------------------------------------------- Jacobian

@pytest.mark.parametrize("mk", [small, medium])
def test_jacobian_matches_complex_step(orc, mk):
    """Analytic Jacobian vs the complex-step derivative of the RHS (no cancellation)."""
    mech = mk()
    m = orc.Mech(mech)
    for y in random_states(mech, 6, 7):
        J = m.jac(y, P_ATM)
        Jc = m.jac_cs(y, P_ATM)
        scale = np.abs(Jc).max(axis=1, keepdims=True) + 1e-300
        err = np.abs(J - Jc) / scale
        assert err.max() < 1e-11, err.max()


# --------------------------------------------------------------------------- LU

@pytest.mark.parametrize("n", [1, 10, 41, 81])
def test_lu_solve_matches_lapack(orc, n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        A = rng.standard_normal((n, n)) + np.eye(n) * rng.uniform(-2, 2)
        b = rng.standard_normal(n)
        x, LU, piv = orc.lu_solve(A, b)
        xr = np.linalg.solve(A, b)
        np.testing.assert_allclose(x, xr, rtol=1e-9, atol=1e-11 * np.abs(xr).max())
        berr = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x))
        assert berr < 1e-14


def test_lu_pivot_ties_take_lowest_row(orc):
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.0, 5.0]])
    x, LU, piv = orc.lu_solve(A, np.array([1.0, 2.0, 3.0]))
    assert piv[0] == 1        # |-3| ties with |3| on rows 1 and 2: row 1 wins
    np.testing.assert_allclose(A @ x, [1.0, 2.0, 3.0], rtol=1e-14)


def test_lu_singular_reports_column(orc):
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    with pytest.raises(np.linalg.LinAlgError):
        orc.lu_solve(A, np.ones(2))


# --------------------------------------------------------------------------- equilibrium

def _equilibrate(m, mech, y0, p=P_ATM):
    """Run the oracle's fast integrator long enough to reach chemical equilibrium."""
    import oracle
    opts = oracle.opts(method=3, rtol=1e-12, max_newton=60, ramp=20)
    y = y0[None, :].copy()
    pp = np.array([p])
    Hs = 1e-9
    for _ in range(44):
        y, st, _ = m.stage_fast(y, pp, None, Hs, Hs / 4, opts, nthreads=1)
        assert st[0] == 0
        Hs *= 2.0
    return y[0]


def test_kinetic_equilibrium_minimises_gibbs_energy(orc):
    """Long-time kinetics reach detailed balance (every q_r -> 0) and the
    equilibrium composition equals the minimum of the ideal-gas mixture Gibbs
    energy G/RT = sum_k n_k (g_k/RT + ln(x_k p / p_atm)) under the element totals
    at the final T and p -- an independent route to the same state."""
    mech = small()
    m = orc.Mech(mech)
    E = mech.elem.T.astype(float)
    assert np.linalg.matrix_rank(np.array([
        np.bincount([i for i in mech.prod[r] if i >= 0], minlength=mech.n_species)
        - np.bincount([i for i in mech.reac[r] if i >= 0], minlength=mech.n_species)
        for r in range(mech.n_reactions)])) == mech.n_species - np.linalg.matrix_rank(E)
    y0 = np.concatenate([np.full(mech.n_species, 1.0 / mech.n_species), [1500.0]])
    y = _equilibrate(m, mech, y0)
    T = y[-1]
    Y = y[:-1]
    rho = P_ATM / (R_U * T * np.sum(Y / mech.W))
    C = rho * Y / mech.W
    kf, kr, Kc = m.rate_coeffs(T, C)
    q, _ = m.progress(T, C)
    fwd = np.array([kf[r] * np.prod([C[i] for i in mech.reac[r] if i >= 0]) for r in range(mech.n_reactions)])
    assert np.all(np.abs(q) <= 1e-8 * fwd)
    # Gibbs minimisation in mole numbers per kg of mixture
    n0 = Y / mech.W
    b = E @ n0
    _, _, _, gRT = m.thermo(T)

    def G(lnn):
        nn = np.exp(lnn)
        return np.sum(nn * (gRT + lnn - np.log(nn.sum()) + np.log(P_ATM / P_ATM)))

    cons = {"type": "eq", "fun": lambda lnn: (E @ np.exp(lnn) - b) / b}
    res = scipy.optimize.minimize(G, np.log(n0), constraints=[cons], method="SLSQP",
                                  options={"ftol": 1e-15, "maxiter": 2000})
    n_eq = np.exp(res.x)
    x_kin = n0 * 0 + C / C.sum()
    x_gibbs = n_eq / n_eq.sum()
    big = x_kin > 1e-6
    np.testing.assert_allclose(x_gibbs[big], x_kin[big], rtol=2e-4)
