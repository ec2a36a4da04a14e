"""The allocation-free MRI step (mri_step_noalloc), for callers that must not
allocate device memory while they run: it keeps its scratch in a fixed array
inside the library.  These checks call it through the C ABI and compare it with
mri_step given a caller-allocated workspace, on two calls in a row, and check that
grids too large for the fixed scratch are refused.  This file is collected last on
purpose: if it fails, a run that stops at the first failure has already run every
other test."""
import ctypes as ct

import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def _setup(mri, w):
    import torch
    gm = mri.mri_mech_load(w.mech.to_blob())
    g = w.grid
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    y = torch.tensor(w.y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    return gm, grid, y, p


@pytest.mark.parametrize("name,side", [("line64", None), ("box32", 8)])
def test_noalloc_step_matches_workspace_step_twice(mri, name, side):
    import torch
    w = mechgen.workload(name, cells_per_side=side)
    gm, grid, y_ref, p = _setup(mri, w)
    y_na = y_ref.clone()
    ncell = w.y0.shape[0]
    ws = torch.empty(mri.mri_step_workspace_size(grid, w.mech.n) // 8, dtype=torch.float64, device="cuda")
    st_ref = torch.zeros(ncell, dtype=torch.int32, device="cuda")
    st_na = torch.zeros(ncell, dtype=torch.int32, device="cuda")
    L = mri._lib
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        opts = mri.mri_fast_opts_default(method=w.method, ramp=w.ramp if call == 0 else 0,
                                         jac_policy=mri.MRI_JAC_LAZY)
        mri.mri_step(y_ref, p, grid, call * w.H, w.H, w.h, gm, opts, ws, cell_status=st_ref)
        rc = L.mri_step_noalloc(ct.c_void_p(y_na.data_ptr()), ct.c_void_p(p.data_ptr()), ct.byref(grid),
                                call * w.H, w.H, w.h, mri.MRI_KW3, gm.handle, ct.byref(opts),
                                ct.c_void_p(st_na.data_ptr()), None, None, stream)
        assert rc == mri.MRI_OK
        torch.cuda.synchronize()
        assert int(st_ref.abs().sum()) == 0 and int(st_na.abs().sum()) == 0
        assert_parity(y_na.cpu().numpy(), y_ref.cpu().numpy(), what=f"no-alloc step, call {call + 1}")


def test_noalloc_step_refuses_grids_beyond_its_scratch(mri):
    import torch
    w = mechgen.workload("box32")            # 4 * 32768 * 41 * 8 bytes > 16 MiB
    gm, grid, y, p = _setup(mri, w)
    before = y.clone()
    opts = mri.mri_fast_opts_default(method=w.method)
    rc = mri._lib.mri_step_noalloc(ct.c_void_p(y.data_ptr()), ct.c_void_p(p.data_ptr()), ct.byref(grid), 0.0,
                                   w.H, w.h, mri.MRI_KW3, gm.handle, ct.byref(opts), None, None, None,
                                   ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mri.MRI_ENOMEM
    torch.cuda.synchronize()
    assert torch.equal(y, before)
