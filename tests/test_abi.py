"""CPU checks of the C ABI: the library loads, exports every entry point that
include/mri.h declares, and rejects bad arguments on the host before any launch."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2211_03293_gb300 as m
    return m


def declared_functions():
    src = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("mri.h", "mri_probe.h", "mri_mlp.h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mri_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mri_stage_fast", "mri_slow_rhs", "mri_step", "mri_mech_load"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mri_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib._lib, n)


def test_binding_names_match_the_header(lib):
    for n in declared_functions():
        assert n in lib.EXPORTED


def test_defaults_and_status_strings(lib):
    o = lib.mri_fast_opts_default()
    assert (o.method, o.newton_rtol, o.newton_atol_Y, o.newton_atol_T, o.max_newton, o.ramp) == (
        3, 1e-10, 1e-20, 1e-10, 10, 0)
    assert (o.jac_policy, o.precision, o.warps_per_block, o.blocks_per_sm, o.time_budget_s) == (0, 0, 0, 0, 0.0)
    assert (o.matrix_cache, o.matrix_cache_bytes) == (None, 0)
    assert (o.adaptive, o.ctrl_rtol, o.ctrl_atol_Y, o.ctrl_atol_T) == (0, 1e-6, 1e-12, 1e-6)
    assert o.newton_safety == 3e-4
    assert (o.schedule, o.lu_variant) == (lib.MRI_SCHED_QUEUE, lib.MRI_LU_AUTO)
    assert lib.mri_status_str(0) == "ok"
    assert "Newton" in lib.mri_status_str(-2)


def test_workspace_size(lib):
    g = lib.grid(32, 32, 32, 1e-4, (1, 1, 1), 1e-5, 4)
    assert lib.mri_step_workspace_size(g, 41) == 4 * 32 ** 3 * 41 * 8
    bad = lib.grid(0, 1, 1, 1e-4, (1, 0, 0), 1e-5, 4)
    assert lib.mri_step_workspace_size(bad, 41) == 0


def test_mech_blob_validation_on_host(lib):
    L = lib._lib
    h = ct.c_void_p()
    assert L.mri_mech_load(b"NOTAMECH" + b"\0" * 64, 72, ct.byref(h)) == lib.MRI_EINVAL
    assert L.mri_mech_load(None, 0, ct.byref(h)) == lib.MRI_EINVAL
    import mechgen
    blob = mechgen.make_mechanism(1000, **mechgen.MECH_SMALL).to_blob()
    assert L.mri_mech_load(blob[:100], 100, ct.byref(h)) == lib.MRI_EINVAL   # truncated


def test_stage_argument_validation_on_host(lib):
    L = lib._lib
    o = lib.mri_fast_opts_default()
    fake = ct.c_void_p(0x1000)   # never dereferenced: the checks fire first
    # null mechanism
    assert L.mri_stage_fast(fake, fake, 4, None, 0, 0.0, 1e-8, 1e-9, None, ct.byref(o), None, None, None,
                            None) == lib.MRI_EINVAL
    bad = lib.mri_fast_opts_default(method=4)
    assert L.mri_stage_fast(fake, fake, 4, None, 0, 0.0, 1e-8, 1e-9, fake, ct.byref(bad), None, None, None,
                            None) == lib.MRI_EINVAL
    for kw in (dict(max_newton=0), dict(max_newton=101), dict(newton_rtol=0.0), dict(ramp=41), dict(precision=7),
               dict(warps_per_block=17), dict(warps_per_block=-1), dict(blocks_per_sm=9),
               dict(time_budget_s=-1.0), dict(time_budget_s=float("nan")), dict(adaptive=2),
               dict(adaptive=1, ctrl_rtol=0.0), dict(adaptive=1, ctrl_atol_T=-1.0), dict(newton_safety=0.0),
               dict(newton_safety=1.5), dict(newton_safety=float("nan")), dict(schedule=2),
               dict(schedule=1, time_budget_s=1.0), dict(lu_variant=5), dict(lu_variant=-1), dict(method=11),
               dict(method=14, adaptive=1), dict(method=15)):
        bad = lib.mri_fast_opts_default(**kw)
        assert L.mri_stage_fast(fake, fake, 4, None, 0, 0.0, 1e-8, 1e-9, fake, ct.byref(bad), None, None, None,
                                None) == lib.MRI_EINVAL
    # the mixed-mechanism launch: group count and launch-shape options are checked first
    grp = (lib.mri_stage_group * 9)()
    assert L.mri_stage_fast_batch(None, 1, 0.0, 1e-8, 1e-9, ct.byref(o), None, None) == lib.MRI_EINVAL
    assert L.mri_stage_fast_batch(grp, 0, 0.0, 1e-8, 1e-9, ct.byref(o), None, None) == lib.MRI_EINVAL
    assert L.mri_stage_fast_batch(grp, 9, 0.0, 1e-8, 1e-9, ct.byref(o), None, None) == lib.MRI_EINVAL
    for kw in (dict(warps_per_block=2), dict(blocks_per_sm=2), dict(time_budget_s=1.0),
               dict(matrix_cache=0x1000, matrix_cache_bytes=1 << 20), dict(schedule=1)):
        bad = lib.mri_fast_opts_default(**kw)
        assert L.mri_stage_fast_batch(grp, 1, 0.0, 1e-8, 1e-9, ct.byref(bad), None, None) == lib.MRI_EINVAL
    # a whole MRI step takes no time budget
    g = lib.grid(4, 1, 1, 1e-4, (1, 0, 0), 1e-5, 2)
    budget = lib.mri_fast_opts_default(time_budget_s=1.0)
    assert L.mri_step(fake, fake, ct.byref(g), 0.0, 1e-7, 1e-9, lib.MRI_KW3, fake, ct.byref(budget), fake,
                      1 << 30, None, None, None, None) == lib.MRI_EINVAL
    g = lib.grid(4, 1, 1, 1e-4, (1, 0, 0), 1e-5, 3)   # order 3 does not exist
    assert L.mri_slow_rhs(fake, fake, 10, ct.byref(g), 0.0, None) == lib.MRI_EINVAL
    assert L.mri_lu_solve_batched(fake, fake, 0, 1, None, None) == lib.MRI_EINVAL
    assert L.mri_lu_solve_batched(fake, fake, 129, 1, None, None) == lib.MRI_EINVAL


def test_imex_and_diffusion_argument_validation_on_host(lib):
    """The implicit-diffusion entry points check their arguments before any launch."""
    L = lib._lib
    fake = ct.c_void_p(0x1000)   # never dereferenced: the checks fire first
    g = lib.grid(8, 8, 8, 1e-4, (1, 0, 0), 1e-5, 2)
    need = L.mri_diffusion_workspace_size(ct.byref(g), 5)
    assert need >= 3 * 8 ** 3 * 5 * 8
    assert L.mri_diffusion_workspace_size(ct.byref(g), 0) == 0
    it = ct.c_int()
    args = dict(a=1e-3, tol=1e-12, max_iter=10, check=8, ws=fake, wsb=need)

    def solve(n=5, **kw):
        a = dict(args, **kw)
        return L.mri_diffusion_solve(fake, fake, n, ct.byref(g), a["a"], a["tol"], a["max_iter"], a["check"],
                                     a["ws"], a["wsb"], ct.byref(it), None, None)
    assert solve(n=0) == lib.MRI_EINVAL
    assert solve(n=1025) == lib.MRI_EINVAL
    assert solve(a=-1.0) == lib.MRI_EINVAL
    assert solve(tol=0.0) == lib.MRI_EINVAL
    assert solve(check=-1) == lib.MRI_EINVAL
    assert solve(wsb=need - 8) == lib.MRI_ENOMEM
    assert solve(ws=None) == lib.MRI_ENOMEM
    o = lib.mri_fast_opts_default()
    assert L.mri_step_imex2(fake, fake, ct.byref(g), 0.0, 1e-7, 1e-9, 7, fake, ct.byref(o), 1e-12, 10, 8, fake,
                            1 << 30, None, None, None, None, None, None) == lib.MRI_EINVAL
    assert L.mri_step_imex1(fake, fake, ct.byref(g), 0.0, -1e-7, 1e-9, fake, ct.byref(o), 1e-12, 10, 8, fake,
                            1 << 30, None, None, None, None, None, None) == lib.MRI_EINVAL
    budget = lib.mri_fast_opts_default(time_budget_s=1.0)
    assert L.mri_step_imex1(fake, fake, ct.byref(g), 0.0, 1e-7, 1e-9, fake, ct.byref(budget), 1e-12, 10, 8, fake,
                            1 << 30, None, None, None, None, None, None) == lib.MRI_EINVAL
    assert L.mri_step_imex2_workspace_size(ct.byref(g), 5) > L.mri_step_imex1_workspace_size(ct.byref(g), 5) > 0

