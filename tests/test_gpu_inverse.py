"""The Gauss-Jordan inverse of MRI_LU_INVERSE: the batched entry point against the
definition of the inverse and the oracle's LU solve, singular and non-finite pivot
columns, and the stage kernel with the inverse variant against the oracle (both
precision forms, the Newton-matrix cache across calls, an entry written by the LU
variant counting as empty)."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nbatch", [(1, 3), (2, 5), (10, 64), (31, 7), (32, 7), (33, 7), (41, 37), (64, 5),
                                      (65, 5), (81, 9), (128, 2)])
def test_batched_inverse(mri, orc, n, nbatch):
    import torch
    rng = np.random.default_rng(n * 7919 + nbatch)
    A = rng.standard_normal((nbatch, n, n)) + np.eye(n) * rng.uniform(-3, 3, (nbatch, 1, 1))
    # Newton-matrix-like systems: I - hg J with a stiff, badly scaled J
    A[0] = np.eye(n) - 1e-9 * rng.standard_normal((n, n)) * 10.0 ** rng.uniform(0, 14, (n, 1))
    if nbatch > 1 and n > 1:
        A[1] = np.roll(np.eye(n), 1, axis=0) * rng.uniform(1, 2, n)[:, None]   # every pivot needs an interchange
    b = rng.standard_normal((nbatch, n))
    Ad, bd = torch.tensor(A, device="cuda"), torch.tensor(b, device="cuda")
    info = torch.full((nbatch,), -7, dtype=torch.int32, device="cuda")
    mri.mri_inverse_solve_batched(Ad, bd, info)
    Ainv, x = Ad.cpu().numpy(), bd.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for s in range(nbatch):
        ref = np.linalg.inv(A[s])
        cond = np.linalg.cond(A[s])
        # forward error of an inverse: cond(A) eps relative to the largest entry
        np.testing.assert_allclose(Ainv[s], ref, rtol=0, atol=64 * n * cond * 2.2e-16 * np.abs(ref).max())
        # A A^-1 = I to the same bound
        eye = A[s] @ Ainv[s]
        assert np.abs(eye - np.eye(n)).max() <= 64 * n * cond * 2.2e-16
        xr, _, _ = orc.lu_solve(A[s], b[s])
        np.testing.assert_allclose(x[s], xr, rtol=0, atol=64 * n * cond * 2.2e-16 * np.abs(xr).max())


def test_batched_inverse_reports_singular_and_nonfinite(mri):
    import torch
    A = torch.tensor([[[1.0, 2.0], [2.0, 4.0]], [[2.0, 0.0], [0.0, 3.0]], [[np.nan, 1.0], [1.0, 1.0]],
                      [[0.0, 1.0], [0.0, 1.0]]], dtype=torch.float64, device="cuda")
    b = torch.ones((4, 2), dtype=torch.float64, device="cuda")
    info = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    mri.mri_inverse_solve_batched(A, b, info)
    assert info.cpu().tolist() == [2, 0, 1, 1]
    np.testing.assert_allclose(b[1].cpu().numpy(), [0.5, 1.0 / 3.0], rtol=1e-15)
    np.testing.assert_allclose(A[1].cpu().numpy(), [[0.5, 0.0], [0.0, 1.0 / 3.0]], rtol=1e-15)


def run_stage(mri, w, y, p, phi, Hs, opts):
    import torch
    gm = mri.mri_mech_load(w.mech.to_blob())
    yd, pd = torch.tensor(y, device="cuda"), torch.tensor(p, device="cuda")
    ph = None if phi is None else torch.tensor(phi, device="cuda")
    st = torch.full((y.shape[0],), -9, dtype=torch.int32, device="cuda")
    ss = torch.zeros((y.shape[0], 4), dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, Hs, w.h, gm, opts, cell_status=st, cell_stats=ss)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy()


@pytest.mark.parametrize("name,method,K,jac,prec", [("line64", 2, 1, 0, 0), ("line64", 2, 2, 1, 1),
                                                    ("box32", 3, 1, 0, 0), ("box32", 3, 0, 1, 0),
                                                    ("box32", 3, 2, 1, 1)])
def test_stage_parity_with_inverse(mri, orc, name, method, K, jac, prec):
    """A first stage with the start-up sequence, full and lazy Jacobians."""
    w = mechgen.workload(name)
    idx = np.sort(np.random.default_rng(31).choice(w.y0.shape[0], min(160, w.y0.shape[0]), replace=False))
    y, p = w.y0[idx], w.p[idx]
    phi = mechgen.random_forcing(12, y.shape[0], w.mech.n, K) if K else None
    o = mri.mri_fast_opts_default(method=method, ramp=w.ramp, jac_policy=jac, precision=prec,
                                  lu_variant=mri.MRI_LU_INVERSE)
    got, st, ss = run_stage(mri, w, y, p, phi, w.H / 3, o)
    ref, rst, _ = orc.Mech(w.mech).stage_fast(y, p, phi, w.H / 3, w.h, orc.opts(method=method, ramp=w.ramp))
    assert np.all(rst == 0) and np.all(st == 0)
    assert_parity(got, ref, what=f"{name} stage, inverse variant, form {prec}")


@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_with_matrix_cache_across_calls(mri, orc, prec):
    """Two calls sharing the cache (the second reuses the first's inverses) against
    the oracle; and a cache written by the LU variant counts as empty for the inverse
    variant: its second call is bitwise the call with a zeroed cache."""
    import torch
    w = mechgen.workload("box32")
    idx = np.sort(np.random.default_rng(32).choice(w.y0.shape[0], 128, replace=False))
    y, p = w.y0[idx], w.p[idx]
    gm = mri.mri_mech_load(w.mech.to_blob())
    phi = mechgen.random_forcing(13, y.shape[0], w.mech.n, 1)
    om = orc.Mech(w.mech)
    r1, st1, _ = om.stage_fast(y, p, phi, w.H / 3, w.h, orc.opts(method=3, ramp=w.ramp))
    r2, st2, _ = om.stage_fast(r1, p, phi, w.H * 5 / 12, w.h, orc.opts(method=3))
    assert np.all(st1 == 0) and np.all(st2 == 0)

    def two_calls(first_variant, second_variant, zero_between=False):
        cache = torch.zeros(mri.mri_matrix_cache_size(gm, y.shape[0], prec), dtype=torch.uint8, device="cuda")
        base = dict(method=3, jac_policy=mri.MRI_JAC_LAZY, precision=prec)
        o1 = mri.with_matrix_cache(mri.mri_fast_opts_default(ramp=w.ramp, lu_variant=first_variant, **base), cache)
        g1, s1, _ = run_stage(mri, w, y, p, phi, w.H / 3, o1)
        if zero_between:
            cache.zero_()
        o2 = mri.with_matrix_cache(mri.mri_fast_opts_default(lu_variant=second_variant, **base), cache)
        g2, s2, ss2 = run_stage(mri, w, g1, p, phi, w.H * 5 / 12, o2)
        assert np.all(s1 == 0) and np.all(s2 == 0)
        return g1, g2, ss2

    inv = mri.MRI_LU_INVERSE
    g1, g2, ss = two_calls(inv, inv)
    assert_parity(g1, r1, what="first call, inverse variant")
    assert_parity(g2, r2, what="second call, cached inverses")
    _, _, ss0 = two_calls(inv, inv, zero_between=True)
    assert ss[:, 2].sum() < ss0[:, 2].sum()   # the cached inverses save Jacobian evaluations
    _, a, _ = two_calls(mri.MRI_LU_AUTO, inv)
    _, b, _ = two_calls(mri.MRI_LU_AUTO, inv, zero_between=True)
    np.testing.assert_array_equal(a, b)
