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
    return {"small": mechgen.make_mechanism(1000, **mechgen.MECH_SMALL),
            "medium": mechgen.make_mechanism(3000, **mechgen.MECH_MEDIUM)}


def states(mech, n, seed):
    rng = np.random.default_rng(seed)
    Y = rng.dirichlet(np.ones(mech.n_species) * rng.choice([0.2, 1.0]), size=n)
    T = rng.uniform(300.0, 2600.0, n)
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


@pytest.mark.parametrize("name", ["small", "medium"])
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


@pytest.mark.parametrize("name", ["small", "medium"])
def test_jacobian_parity(mri, orc, name):
    import torch
    mech = mechs()[name]
    om = orc.Mech(mech)
    gm = mri.mri_mech_load(mech.to_blob())
    y = states(mech, 33, 5)
    p = np.full(33, P_ATM)
    yd = torch.tensor(y, device="cuda")
    pd = torch.tensor(p, device="cuda")
    Jd = torch.zeros((33, mech.n, mech.n), dtype=torch.float64, device="cuda")
    mri.mri_fast_jac(yd, pd, gm, Jd)
    J = Jd.cpu().numpy()
    for c in range(33):
        ref = om.jac(y[c], p[c])
        scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
        err = (np.abs(J[c] - ref) / scale).max()
        assert err < 1e-12, (c, err)


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
