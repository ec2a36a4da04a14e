"""GB300 fast-partition solver for MRI multirate integration of reacting flow.

Thin ctypes binding of ``libmri.so`` (C ABI declared in ``include/mri.h``): the
functions below carry the C names and only marshal arguments.  Every step of
the solve runs in the library's CUDA kernels; there is no CPU fallback, and
importing this package fails loudly when the library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).

Device arrays are passed as CUDA torch tensors (float64 / int32, contiguous);
``stream`` defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmri.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first (paper_2211_03293_gb300/build.py)")

_lib = ct.CDLL(LIB_PATH)

MRI_OK, MRI_EINVAL, MRI_ENEWTON, MRI_ECUDA, MRI_ETIMEOUT, MRI_ENOMEM, MRI_ECONV = 0, -1, -2, -3, -4, -5, -6
MRI_CELL_OK, MRI_CELL_ENEWTON, MRI_CELL_EINPUT, MRI_CELL_TIMEOUT = 0, 1, 2, 3
MRI_SDIRK2, MRI_SDIRK3 = 2, 3
MRI_ERK2, MRI_ERK3, MRI_ERK4 = 12, 13, 14
MRI_KW3 = 1
MRI_JAC_PER_SUBSTEP = 0
MRI_JAC_LAZY = 1
MRI_PREC_FP64 = 0
MRI_PREC_FP32_LU = 1
MRI_START_PREDICTOR, MRI_START_PREVIOUS, MRI_START_GUESS, MRI_START_GUESS_FIRST = 0, 1, 2, 3
MRI_SCHED_QUEUE, MRI_SCHED_STATIC = 0, 1
MRI_LU_AUTO, MRI_LU_REGS, MRI_LU_REGS_SPLIT, MRI_LU_SHARED, MRI_LU_INVERSE = 0, 1, 2, 3, 4


class mri_fast_opts(ct.Structure):
    _fields_ = [("method", ct.c_int), ("newton_rtol", ct.c_double), ("newton_atol_Y", ct.c_double),
                ("newton_atol_T", ct.c_double), ("max_newton", ct.c_int), ("jac_policy", ct.c_int),
                ("precision", ct.c_int), ("ramp", ct.c_int), ("warps_per_block", ct.c_int),
                ("blocks_per_sm", ct.c_int), ("time_budget_s", ct.c_double), ("matrix_cache", ct.c_void_p),
                ("matrix_cache_bytes", ct.c_size_t), ("adaptive", ct.c_int), ("ctrl_rtol", ct.c_double),
                ("ctrl_atol_Y", ct.c_double), ("ctrl_atol_T", ct.c_double), ("newton_safety", ct.c_double),
                ("schedule", ct.c_int), ("lu_variant", ct.c_int)]


class mri_stage_group(ct.Structure):
    _fields_ = [("mech", ct.c_void_p), ("y", ct.c_void_p), ("p", ct.c_void_p), ("ncell", ct.c_int),
                ("phi", ct.c_void_p), ("K", ct.c_int), ("cell_status", ct.c_void_p), ("cell_stats", ct.c_void_p)]


MRI_MAX_GROUPS = 8


class mri_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("dx", ct.c_double),
                ("u", ct.c_double * 3), ("D", ct.c_double), ("order", ct.c_int)]


_vp = ct.c_void_p
_i32p = ct.c_void_p
_lib.mri_mech_load.argtypes = [ct.c_char_p, ct.c_size_t, ct.POINTER(_vp)]
_lib.mri_mech_load.restype = ct.c_int
_lib.mri_mech_free.argtypes = [_vp]
_lib.mri_mech_free.restype = None
_lib.mri_mech_info.argtypes = [_vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
_lib.mri_fast_opts_default.argtypes = [ct.POINTER(mri_fast_opts)]
_lib.mri_fast_opts_default.restype = None
_lib.mri_stage_fast.argtypes = [_vp, _vp, ct.c_int, _vp, ct.c_int, ct.c_double, ct.c_double, ct.c_double, _vp,
                                ct.POINTER(mri_fast_opts), _vp, _vp, _vp, _vp]
_lib.mri_stage_fast_shape.argtypes = [_vp, ct.POINTER(mri_fast_opts), ct.c_int, ct.c_int, ct.POINTER(ct.c_int),
                                      ct.POINTER(ct.c_int), ct.POINTER(ct.c_size_t)]
_lib.mri_stage_fast_batch.argtypes = [ct.POINTER(mri_stage_group), ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                      ct.POINTER(mri_fast_opts), _vp, _vp]
_lib.mri_mlp_create.argtypes = [ct.POINTER(ct.c_int), ct.c_int, ct.c_int, _vp, ct.POINTER(_vp)]
_lib.mri_mlp_free.argtypes = [_vp]
_lib.mri_mlp_free.restype = None
_lib.mri_mlp_num_params.argtypes = [_vp]
_lib.mri_mlp_num_params.restype = ct.c_longlong
_lib.mri_mlp_params.argtypes = [_vp, _vp, _vp]
_lib.mri_mlp_forward.argtypes = [_vp, _vp, ct.c_int, _vp, _vp]
_lib.mri_mlp_grad.argtypes = [_vp, _vp, _vp, _vp, ct.c_int, _vp, _vp, _vp]
_lib.mri_mlp_grad_copy.argtypes = [_vp, _vp, _vp]
_lib.mri_mlp_adam.argtypes = [_vp, ct.c_float, ct.c_int, _vp]
_lib.mri_mlp_status.argtypes = [_vp]
_lib.mri_gemm_bf16.argtypes = [_vp, ct.c_int, _vp, ct.c_int, ct.c_int, ct.c_int, ct.c_int, _vp, ct.c_int, _vp, _vp]
_lib.mri_stage_fast_guided.argtypes = [_vp, _vp, ct.c_int, _vp, ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                       _vp, ct.c_int, ct.c_int, _vp, ct.POINTER(mri_fast_opts), _vp, _vp, _vp, _vp,
                                       _vp, _vp]
_lib.mri_learned_features.argtypes = [_vp, _vp, _vp, ct.c_int, ct.c_int, ct.c_int, ct.c_double, _vp, _vp, _vp,
                                      ct.c_int, _vp]
_lib.mri_learned_targets.argtypes = [_vp, _vp, ct.c_int, ct.c_int, ct.c_int, _vp, _vp, _vp, ct.c_int, _vp]
_lib.mri_learned_guess.argtypes = [_vp, _vp, ct.c_int, ct.c_int, ct.c_int, ct.c_int, _vp, _vp, _vp, _vp]
_lib.mri_learned_moments_workspace_size.argtypes = [ct.c_int]
_lib.mri_learned_moments_workspace_size.restype = ct.c_size_t
_lib.mri_learned_moments.argtypes = [_vp, ct.c_longlong, ct.c_int, ct.c_int, ct.c_float, _vp, _vp, _vp, _vp,
                                     ct.c_size_t, _vp]
_lib.mri_learned_standardise.argtypes = [_vp, ct.c_int, _vp, ct.c_longlong, ct.c_int, _vp, _vp, _vp, ct.c_int, _vp]
_lib.mri_learned_step_targets.argtypes = [_vp, ct.c_int, ct.c_int, ct.c_int, _vp, _vp]
_lib.mri_learned_step_exp.argtypes = [_vp, ct.c_int, ct.c_int, ct.c_int, ct.c_float, ct.c_float, ct.c_int, ct.c_int,
                                      _vp, _vp]
_lib.mri_probe_log.argtypes = [_vp, _vp, ct.c_longlong, _vp]
_lib.mri_probe_exp_pair.argtypes = [_vp, _vp, _vp, ct.c_longlong, _vp]
_lib.mri_matrix_cache_size.argtypes = [_vp, ct.c_int, ct.c_int]
_lib.mri_matrix_cache_size.restype = ct.c_size_t
_lib.mri_diffusion_workspace_size.argtypes = [ct.POINTER(mri_grid), ct.c_int]
_lib.mri_diffusion_workspace_size.restype = ct.c_size_t
_lib.mri_diffusion_solve.argtypes = [_vp, _vp, ct.c_int, ct.POINTER(mri_grid), ct.c_double, ct.c_double, ct.c_int,
                                     ct.c_int, _vp, ct.c_size_t, ct.POINTER(ct.c_int), _vp, _vp]
_lib.mri_step_imex1_workspace_size.argtypes = [ct.POINTER(mri_grid), ct.c_int]
_lib.mri_step_imex1_workspace_size.restype = ct.c_size_t
_lib.mri_step_imex1.argtypes = [_vp, _vp, ct.POINTER(mri_grid), ct.c_double, ct.c_double, ct.c_double, _vp,
                                ct.POINTER(mri_fast_opts), ct.c_double, ct.c_int, ct.c_int, _vp, ct.c_size_t, _vp,
                                _vp, _vp, ct.POINTER(ct.c_int), _vp, _vp]
_lib.mri_step_imex2_workspace_size.argtypes = [ct.POINTER(mri_grid), ct.c_int]
_lib.mri_step_imex2_workspace_size.restype = ct.c_size_t
_lib.mri_step_imex2.argtypes = [_vp, _vp, ct.POINTER(mri_grid), ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                _vp, ct.POINTER(mri_fast_opts), ct.c_double, ct.c_int, ct.c_int, _vp, ct.c_size_t,
                                _vp, _vp, _vp, ct.POINTER(ct.c_int), _vp, _vp]
_lib.mri_slow_rhs.argtypes = [_vp, _vp, ct.c_int, ct.POINTER(mri_grid), ct.c_double, _vp]
_lib.mri_step_workspace_size.argtypes = [ct.POINTER(mri_grid), ct.c_int]
_lib.mri_step_workspace_size.restype = ct.c_size_t
_lib.mri_step.argtypes = [_vp, _vp, ct.POINTER(mri_grid), ct.c_double, ct.c_double, ct.c_double, ct.c_int, _vp,
                          ct.POINTER(mri_fast_opts), _vp, ct.c_size_t, _vp, _vp, _vp, _vp]
_lib.mri_step_noalloc.argtypes = [_vp, _vp, ct.POINTER(mri_grid), ct.c_double, ct.c_double, ct.c_double, ct.c_int,
                                  _vp, ct.POINTER(mri_fast_opts), _vp, _vp, _vp, _vp]
_lib.mri_fast_rhs.argtypes = [_vp, _vp, ct.c_int, _vp, _vp, _vp]
_lib.mri_fast_jac.argtypes = [_vp, _vp, ct.c_int, _vp, _vp, _vp]
_lib.mri_lu_solve_batched.argtypes = [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp]
_lib.mri_inverse_solve_batched.argtypes = [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp]
_lib.mri_stage_forcing.argtypes = [_vp, ct.c_int, ct.c_longlong, ct.POINTER(ct.c_double), _vp, _vp]
_lib.mri_method_coupling.argtypes = [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                     ct.POINTER(ct.c_int)]
_lib.mri_probe_fp64_fma.argtypes = [_vp, ct.c_longlong, ct.c_int, ct.POINTER(ct.c_double), _vp]
_lib.mri_probe_fp64_lanes.argtypes = [_vp, ct.c_longlong, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_double), _vp]
_lib.mri_probe_fp64_latency.argtypes = [_vp, ct.c_longlong, ct.c_int, ct.POINTER(ct.c_double), _vp]
_lib.mri_probe_exp.argtypes = [_vp, _vp, ct.c_longlong, _vp]
_lib.mri_probe_mech_device.argtypes = [_vp, ct.c_int]
_lib.mri_status_str.argtypes = [ct.c_int]
_lib.mri_status_str.restype = ct.c_char_p

EXPORTED = ("mri_mech_load", "mri_mech_free", "mri_mech_info", "mri_fast_opts_default", "mri_stage_fast",
            "mri_slow_rhs", "mri_step_workspace_size", "mri_step", "mri_fast_rhs", "mri_fast_jac",
            "mri_lu_solve_batched", "mri_inverse_solve_batched", "mri_status_str", "mri_stage_forcing", "mri_method_coupling",
            "mri_step_noalloc", "mri_probe_fp64_fma", "mri_probe_fp64_lanes", "mri_probe_fp64_latency", "mri_probe_exp", "mri_stage_fast_shape",
            "mri_stage_fast_batch", "mri_mlp_create", "mri_mlp_free", "mri_mlp_num_params", "mri_mlp_params",
            "mri_mlp_forward", "mri_mlp_grad", "mri_mlp_grad_copy", "mri_mlp_adam", "mri_mlp_status",
            "mri_gemm_bf16", "mri_stage_fast_guided", "mri_learned_features", "mri_learned_targets",
            "mri_learned_guess", "mri_learned_step_exp", "mri_probe_log", "mri_probe_exp_pair",
            "mri_matrix_cache_size", "mri_diffusion_workspace_size", "mri_diffusion_solve",
            "mri_step_imex1_workspace_size", "mri_step_imex1", "mri_step_imex2_workspace_size",
            "mri_step_imex2", "mri_probe_mech_device", "mri_learned_moments_workspace_size",
            "mri_learned_moments", "mri_learned_standardise", "mri_learned_step_targets")


class MriError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {mri_status_str(code)} ({code})")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ct.c_void_p(t.data_ptr())


def _f64(t):
    import torch
    if t is not None and t.dtype != torch.float64:
        raise TypeError("float64 tensor expected")
    return _ptr(t)


def _i32(t):
    import torch
    if t is not None and t.dtype != torch.int32:
        raise TypeError("int32 tensor expected")
    return _ptr(t)


def _i8(t):
    import torch
    if t is not None and t.dtype != torch.int8:
        raise TypeError("int8 tensor expected")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def _check(rc, what):
    if rc != MRI_OK:
        raise MriError(rc, what)
    return rc


def mri_status_str(code: int) -> str:
    return _lib.mri_status_str(code).decode()


def mri_fast_opts_default(**overrides) -> mri_fast_opts:
    o = mri_fast_opts()
    _lib.mri_fast_opts_default(ct.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def grid(nx, ny, nz, dx, u, D, order) -> mri_grid:
    return mri_grid(nx, ny, nz, dx, (ct.c_double * 3)(*u), D, order)


class Mech:
    """Owner of an ``mri_mech`` handle (device tables)."""

    def __init__(self, blob: bytes):
        h = _vp()
        _check(_lib.mri_mech_load(blob, len(blob), ct.byref(h)), "mri_mech_load")
        self.handle = h
        ns, nr = ct.c_int(), ct.c_int()
        _lib.mri_mech_info(h, ct.byref(ns), ct.byref(nr))
        self.n_species, self.n_reactions = ns.value, nr.value
        self.n = self.n_species + 1

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.mri_mech_free(h)
            self.handle = None


def mri_matrix_cache_size(mech: Mech, ncell: int, precision: int = MRI_PREC_FP64) -> int:
    return int(_lib.mri_matrix_cache_size(mech.handle, ncell, precision))


def with_matrix_cache(opts: mri_fast_opts, cache) -> mri_fast_opts:
    """A copy of opts that keeps Newton matrices in `cache` (a zeroed uint8 device
    tensor of mri_matrix_cache_size bytes) between calls."""
    o = mri_fast_opts.from_buffer_copy(opts)
    o.matrix_cache = cache.data_ptr()
    o.matrix_cache_bytes = cache.numel() * cache.element_size()
    return o


def mri_mech_load(blob: bytes) -> Mech:
    return Mech(blob)


def mri_probe_mech_device(mech: Mech, device: int) -> int:
    """Test hook: record `device` as the mechanism's device; returns the previous one."""
    return int(_lib.mri_probe_mech_device(mech.handle, int(device)))


def mri_stage_fast(y, p, phi, t0, Hstage, h, mech: Mech, opts: mri_fast_opts, cell_status=None, cell_stats=None,
                   n_failed=None, stream=None) -> int:
    ncell = y.shape[0]
    K = 0 if phi is None else phi.shape[1]
    rc = _lib.mri_stage_fast(_f64(y), _f64(p), ncell, _f64(phi), K, t0, Hstage, h, mech.handle, ct.byref(opts),
                             _i32(cell_status), _i32(cell_stats), _i32(n_failed), _stream(stream))
    return _check(rc, "mri_stage_fast")


def mri_stage_fast_guided(y, p, phi, t0, Hstage, h, mech: Mech, opts: mri_fast_opts, start=MRI_START_PREDICTOR,
                          guess=None, cell_status=None, cell_stats=None, n_failed=None, n_fallback=None,
                          step_exp=None, stream=None) -> int:
    """mri_stage_fast with a chosen Newton start; guess: [ncell][n_sub][n] float64 (MRI_START_GUESS*);
    step_exp: int8 [ncell], the adaptive first step's power-of-two factor."""
    ncell = y.shape[0]
    K = 0 if phi is None else phi.shape[1]
    G = 0 if guess is None else guess.shape[1]
    rc = _lib.mri_stage_fast_guided(_f64(y), _f64(p), ncell, _f64(phi), K, t0, Hstage, h, _f64(guess), G, start,
                                    mech.handle, ct.byref(opts), _i32(cell_status), _i32(cell_stats), _i32(n_failed),
                                    _i32(n_fallback), _i8(step_exp), _stream(stream))
    return _check(rc, "mri_stage_fast_guided")


def mri_stage_fast_batch(groups, t0, Hstage, h, opts: mri_fast_opts, n_failed=None, stream=None) -> int:
    """One launch over several mechanisms.  groups: sequence of dicts with keys mech
    (Mech), y, p and optionally phi, cell_status, cell_stats (device tensors)."""
    arr = (mri_stage_group * len(groups))()
    for i, g in enumerate(groups):
        phi = g.get("phi")
        arr[i] = mri_stage_group(g["mech"].handle, _f64(g["y"]), _f64(g["p"]), g["y"].shape[0], _f64(phi),
                                 0 if phi is None else phi.shape[1], _i32(g.get("cell_status")),
                                 _i32(g.get("cell_stats")))
    rc = _lib.mri_stage_fast_batch(arr, len(groups), t0, Hstage, h, ct.byref(opts), _i32(n_failed), _stream(stream))
    return _check(rc, "mri_stage_fast_batch")


def mri_stage_fast_shape(mech: Mech, opts: mri_fast_opts, ncell: int, K: int):
    """(warps per CTA, CTAs, shared bytes per CTA) of mri_stage_fast's launch; raises
    MriError if the requested shape does not fit."""
    w, b, s = ct.c_int(), ct.c_int(), ct.c_size_t()
    _check(_lib.mri_stage_fast_shape(mech.handle, ct.byref(opts), ncell, K, ct.byref(w), ct.byref(b), ct.byref(s)),
           "mri_stage_fast_shape")
    return w.value, b.value, s.value


def mri_slow_rhs(y, fS, g: mri_grid, t=0.0, stream=None) -> int:
    return _check(_lib.mri_slow_rhs(_f64(y), _f64(fS), y.shape[1], ct.byref(g), t, _stream(stream)), "mri_slow_rhs")


def mri_step_workspace_size(g: mri_grid, n: int) -> int:
    return _lib.mri_step_workspace_size(ct.byref(g), n)


def mri_step(y, p, g: mri_grid, t, H, h, mech: Mech, opts: mri_fast_opts, workspace, cell_status=None,
             cell_stats=None, n_failed=None, mri_method=MRI_KW3, stream=None) -> int:
    nbytes = workspace.numel() * workspace.element_size()
    rc = _lib.mri_step(_f64(y), _f64(p), ct.byref(g), t, H, h, mri_method, mech.handle, ct.byref(opts),
                       _ptr(workspace), nbytes, _i32(cell_status), _i32(cell_stats), _i32(n_failed),
                       _stream(stream))
    return _check(rc, "mri_step")


def mri_step_noalloc(y, p, g: mri_grid, t, H, h, mech: Mech, opts: mri_fast_opts, cell_status=None,
                     cell_stats=None, n_failed=None, mri_method=MRI_KW3, stream=None) -> int:
    """mri_step with the library's built-in scratch instead of a caller workspace:
    for callers that must not allocate device memory (grids up to 4*ncell*n*8 <= 16 MiB)."""
    rc = _lib.mri_step_noalloc(_f64(y), _f64(p), ct.byref(g), t, H, h, mri_method, mech.handle, ct.byref(opts),
                               _i32(cell_status), _i32(cell_stats), _i32(n_failed), _stream(stream))
    return _check(rc, "mri_step_noalloc")


def mri_diffusion_workspace_size(g: mri_grid, n: int) -> int:
    return int(_lib.mri_diffusion_workspace_size(ct.byref(g), n))


def mri_diffusion_solve(x, b, g: mri_grid, a, workspace, tol=1e-12, max_iter=1000, check_every=8, cg_info=None,
                        stream=None) -> int:
    """(I - a D lap_h) x = b for every component (x: initial guess in, solution out).
    With check_every > 0 returns the CG iterations taken; with check_every = 0 the
    call does not synchronise (graph-capturable) and returns -1, convergence being
    reported in cg_info (device int32[2])."""
    it = ct.c_int(-1)
    rc = _lib.mri_diffusion_solve(_f64(x), _f64(b), x.shape[1], ct.byref(g), float(a), float(tol), int(max_iter),
                                  int(check_every), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                  ct.byref(it), _i32(cg_info), _stream(stream))
    _check(rc, "mri_diffusion_solve")
    return it.value if check_every > 0 else -1


def mri_step_imex1_workspace_size(g: mri_grid, n: int) -> int:
    return int(_lib.mri_step_imex1_workspace_size(ct.byref(g), n))


def mri_step_imex1(y, p, g: mri_grid, t, H, h, mech: Mech, opts: mri_fast_opts, workspace, cg_tol=1e-12,
                   cg_max_iter=1000, cg_check_every=8, cell_status=None, cell_stats=None, n_failed=None,
                   cg_info=None, stream=None) -> int:
    """One first-order IMEX-MRI step; returns the CG iterations of its implicit stage
    (-1 with cg_check_every = 0, which makes the step graph-capturable)."""
    it = ct.c_int(-1)
    rc = _lib.mri_step_imex1(_f64(y), _f64(p), ct.byref(g), t, H, h, mech.handle, ct.byref(opts), float(cg_tol),
                             int(cg_max_iter), int(cg_check_every), _ptr(workspace),
                             workspace.numel() * workspace.element_size(), _i32(cell_status), _i32(cell_stats),
                             _i32(n_failed), ct.byref(it), _i32(cg_info), _stream(stream))
    _check(rc, "mri_step_imex1")
    return it.value if cg_check_every > 0 else -1


def mri_step_imex2_workspace_size(g: mri_grid, n: int) -> int:
    return int(_lib.mri_step_imex2_workspace_size(ct.byref(g), n))


def mri_step_imex2(y, p, g: mri_grid, t, H, h, mech: Mech, opts: mri_fast_opts, workspace, cg_tol=1e-12,
                   cg_max_iter=1000, cg_check_every=8, cell_status=None, cell_stats=None, n_failed=None,
                   cg_info=None, stream=None, method=None) -> int:
    """One second-order Strang-split IMEX multirate step; returns the CG iterations of
    its two diffusion half steps (-1 with cg_check_every = 0)."""
    it = ct.c_int(-1)
    rc = _lib.mri_step_imex2(_f64(y), _f64(p), ct.byref(g), t, H, h, MRI_KW3 if method is None else method,
                             mech.handle, ct.byref(opts), float(cg_tol), int(cg_max_iter), int(cg_check_every),
                             _ptr(workspace), workspace.numel() * workspace.element_size(), _i32(cell_status),
                             _i32(cell_stats), _i32(n_failed), ct.byref(it), _i32(cg_info), _stream(stream))
    _check(rc, "mri_step_imex2")
    return it.value if cg_check_every > 0 else -1


def mri_stage_forcing(fS, nslow, coeffs, phi, stream=None) -> int:
    """phi = sum_j coeffs[j] fS[j]; fS: [>= nslow, ...] device tensor, phi: [...]."""
    c = (ct.c_double * nslow)(*[float(v) for v in coeffs[:nslow]])
    return _check(_lib.mri_stage_forcing(_f64(fS), nslow, phi.numel(), c, _f64(phi), _stream(stream)),
                  "mri_stage_forcing")


def mri_method_coupling(mri_method=MRI_KW3):
    """(c[4], G[4][3]) of the MRI method's MIS-form coupling."""
    c = (ct.c_double * 4)()
    G = (ct.c_double * 12)()
    s = ct.c_int()
    _check(_lib.mri_method_coupling(mri_method, c, G, ct.byref(s)), "mri_method_coupling")
    return list(c)[:s.value], [list(G)[3 * i:3 * i + 3] for i in range(s.value)]


def mri_probe_fp64_fma(scratch, iters=4096, stream=None) -> float:
    """Measured FP64 FMA rate of the current device (FMA/s); scratch: float64 device tensor."""
    rate = ct.c_double()
    rc = _lib.mri_probe_fp64_fma(_f64(scratch), scratch.numel(), iters, ct.byref(rate), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_fp64_fma")
    return rate.value


def mri_probe_fp64_lanes(scratch, active_lanes, warps_per_sm=8, iters=4096, stream=None) -> float:
    """Lane-FMA rate (FMA/s) with only active_lanes lanes of every warp running FP64 FMA
    chains, warps_per_sm warps per SM."""
    rate = ct.c_double()
    rc = _lib.mri_probe_fp64_lanes(_f64(scratch), scratch.numel(), iters, active_lanes, warps_per_sm,
                                   ct.byref(rate), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_fp64_lanes")
    return rate.value


def mri_probe_fp64_latency(scratch, iters=4096, stream=None) -> float:
    """SM cycles per FMA of one dependent FP64 FMA chain in one warp."""
    cyc = ct.c_double()
    rc = _lib.mri_probe_fp64_latency(_f64(scratch), scratch.numel(), iters, ct.byref(cyc), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_fp64_latency")
    return cyc.value


def mri_probe_exp(x, y, stream=None) -> int:
    """y = exp(x) with the kernels' own FP64 exponential (float64 device tensors)."""
    rc = _lib.mri_probe_exp(_f64(x), _f64(y), x.numel(), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_exp")
    return rc


def mri_probe_exp_pair(x, y, z, stream=None) -> int:
    """y = exp(x), z = exp(-x) from the kernels' shared argument reduction."""
    rc = _lib.mri_probe_exp_pair(_f64(x), _f64(y), _f64(z), x.numel(), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_exp_pair")
    return rc


def mri_probe_log(x, y, stream=None) -> int:
    """y = log(x) with the kernels' own FP64 logarithm (float64 device tensors)."""
    rc = _lib.mri_probe_log(_f64(x), _f64(y), x.numel(), _stream(stream))
    if rc != 0:
        raise MriError(rc, "mri_probe_log")
    return rc


def mri_fast_rhs(y, p, mech: Mech, f, stream=None) -> int:
    return _check(_lib.mri_fast_rhs(_f64(y), _f64(p), y.shape[0], mech.handle, _f64(f), _stream(stream)),
                  "mri_fast_rhs")


def mri_fast_jac(y, p, mech: Mech, J, stream=None) -> int:
    return _check(_lib.mri_fast_jac(_f64(y), _f64(p), y.shape[0], mech.handle, _f64(J), _stream(stream)),
                  "mri_fast_jac")


def mri_lu_solve_batched(A, b, info=None, stream=None) -> int:
    return _check(_lib.mri_lu_solve_batched(_f64(A), _f64(b), A.shape[-1], A.shape[0], _i32(info), _stream(stream)),
                  "mri_lu_solve_batched")


def mri_inverse_solve_batched(A, b, info=None, stream=None) -> int:
    return _check(_lib.mri_inverse_solve_batched(_f64(A), _f64(b), A.shape[-1], A.shape[0], _i32(info),
                                                 _stream(stream)), "mri_inverse_solve_batched")


# ----------------------------------------------------------------------------- learned form

def _f32(t):
    import torch
    if t is not None and t.dtype != torch.float32:
        raise TypeError("float32 tensor expected")
    return _ptr(t)


def _bf16(t):
    import torch
    if t is not None and t.dtype != torch.bfloat16:
        raise TypeError("bfloat16 tensor expected")
    return _ptr(t)


class Mlp:
    """Owner of an ``mri_mlp`` handle: network parameters, Adam state and scratch."""

    def __init__(self, dims, batch_max, init_params=None):
        import numpy as np
        d = (ct.c_int * len(dims))(*dims)
        h = _vp()
        buf = None
        if init_params is not None:
            buf = np.ascontiguousarray(init_params, dtype=np.float32)
        rc = _lib.mri_mlp_create(d, len(dims) - 1, batch_max,
                                 None if buf is None else buf.ctypes.data_as(_vp), ct.byref(h))
        _check(rc, "mri_mlp_create")
        self.handle, self.dims, self.batch_max = h, list(dims), batch_max
        self.n_params = _lib.mri_mlp_num_params(h)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.mri_mlp_free(h)
            self.handle = None


def mri_mlp_create(dims, batch_max, init_params=None) -> Mlp:
    return Mlp(dims, batch_max, init_params)


def mri_mlp_free(mlp: Mlp) -> None:
    mlp.__del__()


def mri_mlp_num_params(mlp: Mlp) -> int:
    return int(_lib.mri_mlp_num_params(mlp.handle))


def mri_mlp_params(mlp: Mlp, new=None):
    """The FP32 master parameters (numpy copy); with ``new``, replace them after copying."""
    import numpy as np
    out = np.empty(mlp.n_params, dtype=np.float32)
    src = None if new is None else np.ascontiguousarray(new, dtype=np.float32)
    _check(_lib.mri_mlp_params(mlp.handle, out.ctypes.data_as(_vp), None if src is None else src.ctypes.data_as(_vp)),
           "mri_mlp_params")
    return out


def mri_mlp_forward(mlp: Mlp, x, y, stream=None) -> int:
    return _check(_lib.mri_mlp_forward(mlp.handle, _f32(x), x.shape[0], _f32(y), _stream(stream)), "mri_mlp_forward")


def mri_mlp_grad(mlp: Mlp, x, t, w_out, y, loss=None, stream=None) -> int:
    return _check(_lib.mri_mlp_grad(mlp.handle, _f32(x), _f32(t), _f32(w_out), x.shape[0], _f32(y), _f32(loss),
                                    _stream(stream)), "mri_mlp_grad")


def mri_mlp_grad_copy(mlp: Mlp, dst, stream=None) -> int:
    return _check(_lib.mri_mlp_grad_copy(mlp.handle, _f32(dst), _stream(stream)), "mri_mlp_grad_copy")


def mri_mlp_adam(mlp: Mlp, lr, step, stream=None) -> int:
    return _check(_lib.mri_mlp_adam(mlp.handle, float(lr), int(step), _stream(stream)), "mri_mlp_adam")


def mri_mlp_status(mlp: Mlp) -> int:
    return int(_lib.mri_mlp_status(mlp.handle))


def mri_gemm_bf16(A, B, C, err, stream=None) -> int:
    """C [M][N] fp32 = A [M][K] bf16 @ B [N][K]^T (bf16); err: int32 device flag."""
    M, K = A.shape
    N = B.shape[0]
    return _check(_lib.mri_gemm_bf16(_bf16(A), A.stride(0), _bf16(B), B.stride(0), M, N, K, _f32(C), C.stride(0),
                                     _i32(err), _stream(stream)), "mri_gemm_bf16")


def mri_learned_features(y, p, phi, Hstage, mean, inv_std, x, stream=None) -> int:
    K = 0 if phi is None else phi.shape[1]
    return _check(_lib.mri_learned_features(_f64(y), _f64(p), _f64(phi), K, y.shape[0], y.shape[1], Hstage, _f32(mean),
                                            _f32(inv_std), _f32(x), x.shape[1], _stream(stream)),
                  "mri_learned_features")


def mri_learned_targets(y_in, y_seq, tmean, tinv_std, t, stream=None) -> int:
    return _check(_lib.mri_learned_targets(_f64(y_in), _f64(y_seq), y_seq.shape[1], y_in.shape[0], y_in.shape[1],
                                           _f32(tmean), _f32(tinv_std), _f32(t), t.shape[1], _stream(stream)),
                  "mri_learned_targets")


def mri_learned_moments(X, used, floor_sd, stream=None):
    """Column mean, inverse standard deviation and standard deviation (float32 device
    tensors of `used` values) of the first `used` columns of X [rows][ld] (float32)."""
    import torch
    rows, ld = X.shape
    dev = X.device
    mean = torch.empty(used, dtype=torch.float32, device=dev)
    inv = torch.empty(used, dtype=torch.float32, device=dev)
    sd = torch.empty(used, dtype=torch.float32, device=dev)
    nb = int(_lib.mri_learned_moments_workspace_size(used))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    _check(_lib.mri_learned_moments(_f32(X), rows, used, ld, float(floor_sd), _f32(mean), _f32(inv), _f32(sd),
                                    _ptr(ws), nb, _stream(stream)), "mri_learned_moments")
    return mean, inv, sd


def mri_learned_standardise(X, perm, used, mean, inv_std, out, stream=None) -> int:
    """out[i] = (X[perm[i]] - mean) * inv_std on the first `used` columns, 0 beyond."""
    import torch
    if perm is not None and perm.dtype != torch.int32:
        raise TypeError("int32 permutation expected")
    rows_out = out.shape[0]
    return _check(_lib.mri_learned_standardise(_f32(X), X.shape[1], _ptr(perm), rows_out, int(used), _f32(mean),
                                               _f32(inv_std), _f32(out), out.shape[1], _stream(stream)),
                  "mri_learned_standardise")


def mri_learned_step_targets(accepted, n_sub, k, stride=4, stream=None) -> int:
    """k[c] = log2(n_sub / max(accepted[c * stride], 1)) on the device (accepted: int32)."""
    return _check(_lib.mri_learned_step_targets(_i32(accepted), int(stride), k.shape[0], int(n_sub), _f32(k),
                                                _stream(stream)), "mri_learned_step_targets")


def mri_learned_step_exp(yhat, col, tmean, tstd, step_exp, kmin=-20, kmax=10, stream=None) -> int:
    return _check(_lib.mri_learned_step_exp(_f32(yhat), yhat.shape[1], int(col), yhat.shape[0], float(tmean),
                                            float(tstd), int(kmin), int(kmax), _i8(step_exp), _stream(stream)),
                  "mri_learned_step_exp")


def mri_learned_guess(y_in, yhat, G, tmean, tstd, guess, stream=None) -> int:
    return _check(_lib.mri_learned_guess(_f64(y_in), _f32(yhat), yhat.shape[1], G, y_in.shape[0], y_in.shape[1],
                                         _f32(tmean), _f32(tstd), _f64(guess), _stream(stream)), "mri_learned_guess")
