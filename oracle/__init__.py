"""Python handle on the CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs import this; the CUDA product path
never does.  Every function marshals numpy arrays into the C library, which is
a plain FP64 restatement of the method (see oracle.h for the passages it
follows).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int32)


class Opts(ct.Structure):
    _fields_ = [("method", ct.c_int), ("rtol", ct.c_double), ("atol_Y", ct.c_double),
                ("atol_T", ct.c_double), ("max_newton", ct.c_int), ("ramp", ct.c_int), ("adaptive", ct.c_int),
                ("ctrl_rtol", ct.c_double), ("ctrl_atol_Y", ct.c_double), ("ctrl_atol_T", ct.c_double)]


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("dx", ct.c_double),
                ("u", ct.c_double * 3), ("D", ct.c_double), ("order", ct.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.SO
        if not os.path.exists(path):
            path = _build.build()
        L = ct.CDLL(path)
        L.orc_mech_load.restype = ct.c_void_p
        L.orc_mech_load.argtypes = [ct.c_char_p, ct.c_size_t]
        L.orc_mech_free.argtypes = [ct.c_void_p]
        for name in ("orc_thermo", "orc_rate_coeffs", "orc_progress", "orc_rhs", "orc_jac", "orc_jac_cs",
                     "orc_stage_fast", "orc_mri_step", "orc_single_rate", "orc_mech_info"):
            getattr(L, name).argtypes = None
        L.orc_thermo.argtypes = [ct.c_void_p, ct.c_double, _dp, _dp, _dp, _dp]
        L.orc_rate_coeffs.argtypes = [ct.c_void_p, ct.c_double, _dp, _dp, _dp, _dp]
        L.orc_progress.argtypes = [ct.c_void_p, ct.c_double, _dp, _dp, _dp]
        L.orc_rhs.argtypes = [ct.c_void_p, _dp, ct.c_double, _dp]
        L.orc_jac.argtypes = [ct.c_void_p, _dp, ct.c_double, _dp]
        L.orc_jac_cs.argtypes = [ct.c_void_p, _dp, ct.c_double, _dp]
        L.orc_mech_info.argtypes = [ct.c_void_p, _ip, _ip]
        L.orc_lu_solve.argtypes = [ct.c_int, _dp, _ip, _dp]
        L.orc_flop_counts.argtypes = [ct.c_void_p, _dp, ct.c_double, ct.c_double, ct.POINTER(ct.c_longlong)]
        L.orc_sdirk_tableau.argtypes = [ct.c_int, _dp, _dp, _dp, _ip]
        L.orc_mri_tableau.argtypes = [_dp, _dp, _ip]
        L.orc_erk_tableau.argtypes = [ct.c_int, _dp, _dp, _dp, _ip]
        L.orc_erk_scalar.argtypes = [ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                     ct.c_double, _dp]
        L.orc_mri_coupling.argtypes = [_dp, _ip]
        L.orc_stage_fast.argtypes = [ct.c_void_p, _dp, _dp, ct.c_int, _dp, ct.c_int, ct.c_double, ct.c_double,
                                     ct.POINTER(Opts), _ip, _ip, ct.c_int]
        L.orc_stage_fast_exp.argtypes = [ct.c_void_p, _dp, _dp, ct.c_int, _dp, ct.c_int, ct.c_double,
                                         ct.c_double, ct.POINTER(Opts), ct.c_void_p, _ip, _ip, ct.c_int]
        L.orc_slow_rhs.argtypes = [_dp, _dp, ct.c_int, ct.POINTER(Grid)]
        L.orc_mri_step.argtypes = [ct.c_void_p, _dp, _dp, ct.POINTER(Grid), ct.c_double, ct.c_double,
                                   ct.POINTER(Opts), _ip, _ip, ct.c_int]
        L.orc_single_rate.argtypes = [ct.c_void_p, _dp, _dp, ct.POINTER(Grid), ct.c_double, ct.c_int,
                                      ct.POINTER(Opts)]
        L.orc_sdirk_scalar.argtypes = [ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                       ct.c_double, _dp]
        L.orc_kpr_mri.argtypes = [ct.c_int, ct.c_double, ct.c_double, ct.c_double, ct.c_double, ct.c_double,
                                  ct.c_int, ct.c_int, _dp, _dp]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def opts(method=3, rtol=1e-10, atol_Y=1e-20, atol_T=1e-10, max_newton=10, ramp=0, adaptive=0, ctrl_rtol=1e-6,
         ctrl_atol_Y=1e-12, ctrl_atol_T=1e-6) -> Opts:
    return Opts(method, rtol, atol_Y, atol_T, max_newton, ramp, adaptive, ctrl_rtol, ctrl_atol_Y, ctrl_atol_T)


def grid(g: dict) -> Grid:
    return Grid(g["nx"], g["ny"], g["nz"], g["dx"], (ct.c_double * 3)(*g["u"]), g["D"], g["order"])


def default_threads() -> int:
    return os.cpu_count() or 1


class Mech:
    """An oracle-side mechanism parsed from a mechgen blob."""

    def __init__(self, mechanism):
        blob = mechanism.to_blob() if hasattr(mechanism, "to_blob") else bytes(mechanism)
        self._blob = blob
        self.ptr = lib().orc_mech_load(blob, len(blob))
        if not self.ptr:
            raise ValueError("oracle rejected the mechanism blob")
        ns, nr = ct.c_int32(), ct.c_int32()
        lib().orc_mech_info(self.ptr, ct.byref(ns), ct.byref(nr))
        self.Ns, self.R = ns.value, nr.value
        self.n = self.Ns + 1

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_mech_free(self.ptr)
            self.ptr = None

    def thermo(self, T):
        out = [np.zeros(self.Ns) for _ in range(4)]
        rc = lib().orc_thermo(self.ptr, float(T), *[_d(o) for o in out])
        assert rc == 0
        return tuple(out)   # cp/R, h/RT, s/R, g/RT

    def rate_coeffs(self, T, C):
        kf, kr, Kc = np.zeros(self.R), np.zeros(self.R), np.zeros(self.R)
        C = _f64(C)
        assert lib().orc_rate_coeffs(self.ptr, float(T), _d(C), _d(kf), _d(kr), _d(Kc)) == 0
        return kf, kr, Kc

    def progress(self, T, C):
        q, w = np.zeros(self.R), np.zeros(self.Ns)
        C = _f64(C)
        assert lib().orc_progress(self.ptr, float(T), _d(C), _d(q), _d(w)) == 0
        return q, w

    def rhs(self, y, p):
        y = _f64(y)
        f = np.zeros(self.n)
        assert lib().orc_rhs(self.ptr, _d(y), float(p), _d(f)) == 0
        return f

    def jac(self, y, p):
        y = _f64(y)
        J = np.zeros((self.n, self.n))
        assert lib().orc_jac(self.ptr, _d(y), float(p), _d(J)) == 0
        return J

    def flop_counts(self, y, p, hg):
        """Operation counts of the oracle's formulas at state y: a dict of rows (rhs, jac,
        lu, solve), each a dict of categories (add, mul, div, exp, log, pow)."""
        y = _f64(y)
        out = (ct.c_longlong * 24)()
        assert lib().orc_flop_counts(self.ptr, _d(y), float(p), float(hg), out) == 0
        cats = ("add", "mul", "div", "exp", "log", "pow")
        return {row: {c: int(out[6 * i + j]) for j, c in enumerate(cats)}
                for i, row in enumerate(("rhs", "jac", "lu", "solve"))}

    def jac_cs(self, y, p):
        y = _f64(y)
        J = np.zeros((self.n, self.n))
        assert lib().orc_jac_cs(self.ptr, _d(y), float(p), _d(J)) == 0
        return J

    def stage_fast(self, y, p, phi, Hs, h, o: Opts, nthreads=None, step_exp=None):
        """One MRI stage's fast IVP for every cell; returns (y_new, status, stats).
        step_exp (int8 per cell, adaptive mode): first step = uniform substep * 2^k."""
        y = _f64(y).copy()
        ncell = y.shape[0]
        p = _f64(p)
        phi = _f64(phi) if phi is not None else None
        K = phi.shape[1] if phi is not None else 0
        status = np.zeros(ncell, np.int32)
        stats = np.zeros((ncell, 4), np.int32)
        if step_exp is None:
            rc = lib().orc_stage_fast(self.ptr, _d(y), _d(p), ncell, _d(phi), K, float(Hs), float(h),
                                      ct.byref(o), _i(status), _i(stats), nthreads or default_threads())
        else:
            ke = np.ascontiguousarray(step_exp, dtype=np.int8)
            assert ke.shape == (ncell,)
            rc = lib().orc_stage_fast_exp(self.ptr, _d(y), _d(p), ncell, _d(phi), K, float(Hs), float(h),
                                          ct.byref(o), ke.ctypes.data_as(ct.c_void_p), _i(status), _i(stats),
                                          nthreads or default_threads())
        if rc < 0:
            raise ValueError("orc_stage_fast rejected its arguments")
        return y, status, stats

    def mri_step(self, y, p, g: dict, H, h, o: Opts, nthreads=None):
        y = _f64(y).copy()
        ncell = y.shape[0]
        status = np.zeros(ncell, np.int32)
        stats = np.zeros((ncell, 4), np.int32)
        gr = grid(g)
        rc = lib().orc_mri_step(self.ptr, _d(y), _d(_f64(p)), ct.byref(gr), float(H), float(h), ct.byref(o),
                                _i(status), _i(stats), nthreads or default_threads())
        if rc < 0:
            raise ValueError("orc_mri_step rejected its arguments")
        return y, status, stats

    def single_rate(self, y, p, g: dict, t_end, nsteps, o: Opts):
        y = _f64(y).copy()
        gr = grid(g)
        rc = lib().orc_single_rate(self.ptr, _d(y), _d(_f64(p)), ct.byref(gr), float(t_end), int(nsteps),
                                   ct.byref(o))
        if rc != 0:
            raise RuntimeError(f"orc_single_rate failed ({rc})")
        return y


def lu_solve(A, b):
    A = _f64(A).copy()
    b = _f64(b).copy()
    n = A.shape[0]
    piv = np.zeros(n, np.int32)
    rc = lib().orc_lu_solve(n, _d(A), _i(piv), _d(b))
    if rc != 0:
        raise np.linalg.LinAlgError(f"singular at column {rc - 1}")
    return b, A, piv


def sdirk_tableau(method):
    A, b, c, s = np.zeros(9), np.zeros(3), np.zeros(3), ct.c_int32()
    assert lib().orc_sdirk_tableau(method, _d(A), _d(b), _d(c), ct.byref(s)) == 0
    s = s.value
    return A[: s * s].reshape(s, s), b[:s], c[:s]


def sdirk_embedded(method):
    """(bhat, q): embedded weights of the adaptive controller's error estimate."""
    bhat, q = np.zeros(3), ct.c_int32()
    assert lib().orc_sdirk_embedded(method, _d(bhat), ct.byref(q)) == 0
    return bhat[:method], q.value


def erk_tableau(method):
    """(A, b, c) of the explicit fast method 12 (Heun), 13 (Kutta 3) or 14 (RK4)."""
    A, b, c, s = np.zeros(16), np.zeros(4), np.zeros(4), ct.c_int32()
    assert lib().orc_erk_tableau(method, _d(A), _d(b), _d(c), ct.byref(s)) == 0
    s = s.value
    return A[: s * s].reshape(s, s), b[:s], c[:s]


def erk_scalar(method, problem, lam, t0, t1, nsteps, y0):
    out = np.zeros(1)
    if lib().orc_erk_scalar(method, problem, lam, t0, t1, nsteps, y0, _d(out)) != 0:
        raise RuntimeError("explicit scalar integration failed")
    return out[0]


def mri_tableau():
    A, c, s = np.zeros(16), np.zeros(4), ct.c_int32()
    lib().orc_mri_tableau(_d(A), _d(c), ct.byref(s))
    return A.reshape(4, 4), c


def mri_coupling():
    G, s = np.zeros(16), ct.c_int32()
    lib().orc_mri_coupling(_d(G), ct.byref(s))
    return G.reshape(4, 4)


def slow_rhs(y, g: dict):
    y = _f64(y)
    f = np.zeros_like(y)
    gr = grid(g)
    assert lib().orc_slow_rhs(_d(y), _d(f), y.shape[1], ct.byref(gr)) == 0
    return f


def diffusion_solve(b, g: dict, a):
    """Exact solution of (I - a D lap_h) x = b on the periodic grid (lap_h the 7-point
    second-order Laplacian; axes with one cell skipped): the discrete Fourier transform
    diagonalises lap_h with eigenvalues -sum_axes (4/dx^2) sin^2(pi k / N)."""
    b = _f64(b)
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    n = b.shape[1]
    B = b.reshape(nz, ny, nx, n)
    lam = np.zeros((nz, ny, nx))
    for axis, N in ((2, nx), (1, ny), (0, nz)):
        if N == 1:
            continue
        s2 = (4.0 / g["dx"] ** 2) * np.sin(np.pi * np.arange(N) / N) ** 2
        shape = [1, 1, 1]
        shape[axis] = N
        lam = lam + s2.reshape(shape)
    X = np.fft.ifftn(np.fft.fftn(B, axes=(0, 1, 2)) / (1.0 + a * g["D"] * lam)[..., None], axes=(0, 1, 2))
    return np.ascontiguousarray(X.real.reshape(-1, n))


def imex1_step(mech: "Mech", y, p, g: dict, H, h, o: Opts):
    """One first-order solve-decoupled IMEX-MRI step: the fast stage over [0, H] with
    the constant forcing f^E(y_n) + f^I(y_n) (f^E the grid's advection, f^I = D lap_h y
    with the 7-point Laplacian), then (I - H L) y_{n+1} = v - H L y_n solved exactly.
    Returns (y_{n+1}, status, stats)."""
    gE = dict(g, D=0.0)
    gI = dict(g, u=(0.0, 0.0, 0.0), order=2)
    fE = slow_rhs(y, gE)
    fI = slow_rhs(y, gI)
    v, st, ss = mech.stage_fast(y, p, (fE + fI)[:, None, :], H, h, o)
    return diffusion_solve(v - H * fI, gI, H), st, ss


def imex2_step(mech: "Mech", y, p, g: dict, H, h, o: Opts):
    """One second-order Strang-split IMEX multirate step: a Crank-Nicolson half step
    of the diffusion, (I - (H/4) L) y* = (I + (H/4) L) y_n (L = D lap_h, 7-point), the
    MRI3 step over H with the chemistry fast and the advection (the grid with D = 0)
    as the explicit slow partition, and a second Crank-Nicolson half step.  Returns
    (y_{n+1}, status, stats)."""
    gE = dict(g, D=0.0)
    gI = dict(g, u=(0.0, 0.0, 0.0), order=2)
    a = H / 4.0
    y1 = diffusion_solve(_f64(y) + a * slow_rhs(y, gI), gI, a)
    y2, st, ss = mech.mri_step(y1, p, gE, H, h, o)
    return diffusion_solve(y2 + a * slow_rhs(y2, gI), gI, a), st, ss


def sdirk_scalar(method, problem, lam, t0, t1, nsteps, y0):
    out = np.zeros(1)
    rc = lib().orc_sdirk_scalar(method, problem, lam, t0, t1, nsteps, y0, _d(out))
    if rc != 0:
        raise RuntimeError("scalar SDIRK failed")
    return out[0]


def kpr_mri(fast_method, G, e, beta, omega, t1, nsteps, m_fast):
    err = np.zeros(1)
    yo = np.zeros(2)
    rc = lib().orc_kpr_mri(fast_method, G, e, beta, omega, t1, nsteps, m_fast, _d(err), _d(yo))
    if rc != 0:
        raise RuntimeError("KPR MRI failed")
    return err[0], yo
