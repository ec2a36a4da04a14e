"""GPU parity of the separate kernels of the fast path (rates / RHS, Jacobian,
batched LU) and of the slow-partition stencil, against the CPU oracle on the same
seeded inputs, called through the C ABI."""
import numpy as np
import pytest

import mechgen

pytestmark = pytest.mark.gpu

R_U = 8.314462618
P_ATM = 101325.0


def mechs():
    # "tb32" and "tb33": 32 and 33 third-body and falloff reactions, the edge of the
    # rate kernel's split between its general first slot and its plain-reaction code
    # (all of them in the first 32 reactions, or not); "large" has 40
    return {"small": mechgen.make_mechanism(1000, **mechgen.MECH_SMALL),
            "medium": mechgen.make_mechanism(3000, **mechgen.MECH_MEDIUM),
            "tb32": mechgen.make_mechanism(3100, **dict(mechgen.MECH_MEDIUM, n_thirdbody=24, n_troe=8)),
            "tb33": mechgen.make_mechanism(3200, **dict(mechgen.MECH_MEDIUM, n_thirdbody=25, n_troe=8)),
            "large": mechgen.make_mechanism(5000, **mechgen.MECH_LARGE)}


def states(mech, n, seed, tmin=300.0):
    rng = np.random.default_rng(seed)
    Y = rng.dirichlet(np.ones(mech.n_species) * rng.choice([0.2, 1.0]), size=n)
    T = rng.uniform(tmin, 2600.0, n)
    return np.concatenate([Y, T[:, None]], axis=1)


def gross_rhs_scale(om, mech, y, p):
    """Size of the terms that cancel in f^F: for every species W_k/rho times
    sum_r |nu_kr| [M]_r (|k_f prod C^nu'| + |k_r prod C^nu''|) -- forward and reverse
    rates cancel inside q_r near partial equilibrium -- and for T the same sums
    weighted by |h_k/RT| times T/(rho cp).  Rounding bounds scale with these."""
    T = y[-1]
    S = np.sum(y[:-1] / mech.W)
    rho = p / (R_U * T * S)
    C = rho * y[:-1] / mech.W
    kf, kr, _ = om.rate_coeffs(T, C)
    gross = np.zeros(mech.n_species)
    for r in range(mech.n_reactions):
        fwd = np.prod([C[i] for i in mech.reac[r] if i >= 0])
        rev = np.prod([C[i] for i in mech.prod[r] if i >= 0])
        term = abs(kf[r] * fwd) + abs(kr[r] * rev)
        if mech.rtype[r] == 1:
            term *= np.dot(mech.eff[mech.eff_row[r]], C)
        for i in list(mech.reac[r]) + list(mech.prod[r]):
            if i >= 0:
                gross[i] += term
    cp, hRT, _, _ = om.thermo(T)
    cpm = np.sum(y[:-1] * cp / mech.W)
    gT = T / (rho * cpm) * np.sum(np.abs(hRT) * gross)
    return np.concatenate([gross * mech.W / rho, [gT]])


@pytest.mark.parametrize("name", ["small", "medium", "tb32", "tb33", "large"])
def test_rhs_parity(mri, orc, name):
    import torch
    mech = mechs()[name]
    om = orc.Mech(mech)
    gm = mri.mri_mech_load(mech.to_blob())
    y = states(mech, 77, 11)          # ragged: not a multiple of the warps per CTA
    p = np.full(77, P_ATM) * np.random.default_rng(2).uniform(0.5, 2.0, 77)
    yd = torch.tensor(y, device="cuda")
    pd = torch.tensor(p, device="cuda")
    fd = torch.zeros_like(yd)
    mri.mri_fast_rhs(yd, pd, gm, fd)
    f = fd.cpu().numpy()
    # rate coefficients are exponentials of arguments of size ~10..100 whose rounding
    # differs between the two implementations: ~1e-14 relative on every rate term
    worst = 0.0
    for c in range(77):
        ref = om.rhs(y[c], p[c])
        scale = gross_rhs_scale(om, mech, y[c], p[c])
        worst = max(worst, float(np.max(np.abs(f[c] - ref) / (scale + 1e-300))))
    assert worst <= 1e-12, worst


def gross_jac_scale(om, mech, y, p):
    """Size of the terms that cancel in the species block of the Jacobian,
    J_kj = (W_k / W_j) (D_kj - (DC_k - wdot_k) / (rho S)), D = sum_r nu_r dq_r/dC: for
    every entry the same formula with every term taken by its magnitude -- forward and
    reverse contributions of a reaction, and of different reactions, cancel near
    partial equilibrium, where rounding bounds scale with these sums, not with J."""
    T = y[-1]
    S = np.sum(y[:-1] / mech.W)
    rho = p / (R_U * T * S)
    C = rho * y[:-1] / mech.W
    kf, kr, _ = om.rate_coeffs(T, C)
    Ns = mech.n_species
    Dg = np.zeros((Ns, Ns))
    wg = np.zeros(Ns)
    for r in range(mech.n_reactions):
        re = [i for i in mech.reac[r] if i >= 0]
        pr = [i for i in mech.prod[r] if i >= 0]
        M = float(np.dot(mech.eff[mech.eff_row[r]], C)) if mech.rtype[r] != 0 else 1.0
        wM = M if mech.rtype[r] == 1 else 1.0
        fwd, rev = abs(kf[r] * np.prod(C[re])), abs(kr[r] * np.prod(C[pr]))
        g = np.zeros(Ns)
        for lst, k in ((re, abs(kf[r])), (pr, abs(kr[r]))):
            for j in range(len(lst)):
                g[lst[j]] += wM * k * np.prod([C[lst[jj]] for jj in range(len(lst)) if jj != j])
        if mech.rtype[r] != 0:      # d[M]/dC through the efficiencies (falloff: d ln k_f / d[M] ~ 1/[M])
            g += np.abs(mech.eff[mech.eff_row[r]]) * (fwd + rev) / (1.0 if mech.rtype[r] == 1 else M)
        for i in set(re + pr):
            nu = abs(pr.count(i) - re.count(i))
            Dg[i] += nu * g
            wg[i] += nu * wM * (fwd + rev)
    DCg = Dg @ C
    return (mech.W[:, None] / mech.W[None, :]) * (Dg + ((DCg + wg) / (rho * S))[:, None])


# The larger mechanisms at flame temperatures (the paper's regime), at 1e-11: their
# Jacobians carry more cancellation, and on cold random states even the oracle's own
# analytic and complex-step evaluations part by more than 1e-12 of the term sizes.
@pytest.mark.parametrize("name,rtol,tmin", [("small", 1e-12, 300.0), ("medium", 1e-12, 300.0),
                                            ("tb32", 1e-11, 1000.0), ("tb33", 1e-11, 1000.0),
                                            ("large", 1e-11, 1000.0)])
def test_jacobian_parity(mri, orc, name, rtol, tmin):
    import torch
    mech = mechs()[name]
    om = orc.Mech(mech)
    gm = mri.mri_mech_load(mech.to_blob())
    y = states(mech, 33, 5, tmin)
    p = np.full(33, P_ATM)
    yd = torch.tensor(y, device="cuda")
    pd = torch.tensor(p, device="cuda")
    Jd = torch.zeros((33, mech.n, mech.n), dtype=torch.float64, device="cuda")
    mri.mri_fast_jac(yd, pd, gm, Jd)
    J = Jd.cpu().numpy()
    Ns = mech.n_species
    for c in range(33):
        ref = om.jac(y[c], p[c])
        # Row by row: the largest difference in a row within rtol of the row's largest
        # cancelling-term size, or within 4 times the largest distance in that row between
        # the oracle's two evaluations of it (analytic and complex step), whichever is
        # larger.  Rounding errors of a row come mostly from its common terms (the mixing
        # term (DC_k - wdot_k) / (rho S) and the third-body sums): in the larger
        # mechanisms and at low temperatures these are sums whose terms cancel beyond what
        # the term sizes show, and there any two FP64 evaluations differ.  The temperature
        # row and column are held to their rows' largest entries the same way.
        cs = om.jac_cs(y[c], p[c])
        gross = gross_jac_scale(om, mech, y[c], p[c])
        d_gpu = np.abs(J[c] - ref)
        d_orc = np.abs(cs - ref)
        scale = np.abs(ref).max(axis=1) + 1e-300
        for k in range(mech.n):
            cols = slice(0, Ns) if k < Ns else slice(0, mech.n)
            size = gross[k].max() if k < Ns else scale[k]
            tol = max(rtol * size, 4.0 * d_orc[k, cols].max())
            assert d_gpu[k, cols].max() <= tol, (c, k, d_gpu[k, cols].max(), tol)
        tol_T = np.maximum(rtol * scale, 4.0 * d_orc[:, Ns])
        assert np.all(d_gpu[:, Ns] <= tol_T), (c, "temperature column")


@pytest.mark.parametrize("n,nbatch", [(1, 3), (10, 64), (41, 37), (81, 9), (128, 2)])
def test_batched_lu_parity(mri, orc, n, nbatch):
    import torch
    rng = np.random.default_rng(n * 1000 + nbatch)
    A = rng.standard_normal((nbatch, n, n)) + np.eye(n) * rng.uniform(-3, 3, (nbatch, 1, 1))
    # Newton-matrix-like systems: I - hg J with a stiff, badly scaled J
    A[0] = np.eye(n) - 1e-9 * rng.standard_normal((n, n)) * 10.0 ** rng.uniform(0, 14, (n, 1))
    b = rng.standard_normal((nbatch, n))
    Ad = torch.tensor(A, device="cuda")
    bd = torch.tensor(b, device="cuda")
    info = torch.zeros(nbatch, dtype=torch.int32, device="cuda")
    mri.mri_lu_solve_batched(Ad, bd, info)
    x = bd.cpu().numpy()
    LU = Ad.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for s in range(nbatch):
        xr, LUr, piv = orc.lu_solve(A[s], b[s])
        np.testing.assert_allclose(LU[s], LUr, rtol=0, atol=1e-12 * np.abs(LUr).max())
        berr = np.linalg.norm(A[s] @ x[s] - b[s]) / (np.linalg.norm(A[s], 2) * np.linalg.norm(x[s]))
        assert berr < 1e-14
        np.testing.assert_allclose(x[s], xr, rtol=0, atol=1e-8 * np.abs(xr).max())


def test_batched_lu_reports_singular(mri):
    import torch
    A = torch.tensor([[[1.0, 2.0], [2.0, 4.0]], [[2.0, 0.0], [0.0, 3.0]]], dtype=torch.float64, device="cuda")
    b = torch.ones((2, 2), dtype=torch.float64, device="cuda")
    info = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    mri.mri_lu_solve_batched(A, b, info)
    assert info.cpu().tolist() == [2, 0]
    np.testing.assert_allclose(b[1].cpu().numpy(), [0.5, 1.0 / 3.0], rtol=1e-15)


@pytest.mark.parametrize("shape,order", [((64, 1, 1), 2), ((5, 3, 7), 4), ((32, 32, 32), 4), ((9, 1, 4), 2)])
def test_slow_rhs_parity(mri, orc, shape, order):
    import torch
    nx, ny, nz = shape
    n = 10
    rng = np.random.default_rng(nx * ny * nz)
    y = rng.uniform(0.0, 1.0, (nx * ny * nz, n))
    y[:, -1] = rng.uniform(300, 2500, nx * ny * nz)
    g = dict(nx=nx, ny=ny, nz=nz, dx=1e-4, u=(1.0, -0.5, 0.25), D=1e-5, order=order)
    ref = orc.slow_rhs(y, g)
    yd = torch.tensor(y, device="cuda")
    fd = torch.zeros_like(yd)
    mri.mri_slow_rhs(yd, fd, mri.grid(nx, ny, nz, 1e-4, (1.0, -0.5, 0.25), 1e-5, order))
    f = fd.cpu().numpy()
    # rounding of a stencil scales with sum |w| max |y| (the terms that cancel)
    wsum = 3 * (abs(1.0) / 1e-4 + 4 * 1e-5 / 1e-8) * 2
    tol = 1e-14 * wsum * np.abs(y).max(axis=0)
    assert np.all(np.abs(f - ref) <= tol)
