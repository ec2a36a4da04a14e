"""The implicit diffusion solve (Jacobi-PCG on the 7-point Laplacian) and the
first-order IMEX-MRI step on the GPU against the oracle's exact Fourier solve and
its IMEX step."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,a", [((32, 32, 32), 3e-3), ((64, 1, 1), 1e-2), ((9, 7, 5), 3e-4)])
def test_diffusion_solve_matches_fourier_solution(mri, orc, shape, a):
    import torch
    nx, ny, nz = shape
    n = 41
    g = dict(nx=nx, ny=ny, nz=nz, dx=1e-4, u=(0.0, 0.0, 0.0), D=1e-5, order=2)
    grid = mri.grid(nx, ny, nz, 1e-4, (0.0, 0.0, 0.0), 1e-5, 2)
    rng = np.random.default_rng(nx + 10 * ny + 100 * nz)
    b = rng.standard_normal((nx * ny * nz, n)) * 10.0 ** rng.uniform(-3, 3, n)
    ref = orc.diffusion_solve(b, g, a)
    bd = torch.tensor(b, device="cuda")
    xd = bd.clone()                              # initial guess: b
    ws = torch.empty(mri.mri_diffusion_workspace_size(grid, n), dtype=torch.uint8, device="cuda")
    its = mri.mri_diffusion_solve(xd, bd, grid, a, ws, tol=1e-13, max_iter=2000)
    x = xd.cpu().numpy()
    err = np.abs(x - ref) / np.abs(ref).max(axis=0)
    assert err.max() < 1e-11, err.max()
    assert 0 < its < 2000


def test_diffusion_solve_reports_no_convergence(mri):
    import torch
    grid = mri.grid(32, 32, 1, 1e-4, (0.0, 0.0, 0.0), 1e-5, 2)
    b = torch.rand((32 * 32, 3), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    ws = torch.empty(mri.mri_diffusion_workspace_size(grid, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(mri.MriError) as e:
        mri.mri_diffusion_solve(x, b, grid, 1.0, ws, tol=1e-14, max_iter=2)
    assert e.value.code == mri.MRI_ECONV


@pytest.mark.parametrize("name,cells", [("line64", None), ("box32", 8)])
def test_imex1_step_matches_oracle(mri, orc, name, cells):
    import torch
    w = mechgen.workload(name, cells_per_side=cells)
    g = dict(w.grid, D=w.grid["D"] * 200)       # H D / dx^2 about 1e-2: several CG iterations
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    m = orc.Mech(w.mech)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, w.H / 3, w.h, orc.opts(method=w.method, ramp=w.ramp))
    H = w.H / 2
    ref, rst, _ = orc.imex1_step(m, y0, w.p, g, H, w.h, orc.opts(method=w.method))
    assert np.all(rst == 0)
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.tensor(y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    st = torch.zeros(y0.shape[0], dtype=torch.int32, device="cuda")
    ws = torch.empty(mri.mri_step_imex1_workspace_size(grid, w.mech.n), dtype=torch.uint8, device="cuda")
    its = mri.mri_step_imex1(y, p, grid, 0.0, H, w.h, gm, mri.mri_fast_opts_default(method=w.method, jac_policy=1),
                             ws, cg_tol=1e-14, cell_status=st)
    assert int((st != 0).sum()) == 0 and its > 0
    assert_parity(y.cpu().numpy(), ref, what=f"IMEX1 step {name}")


def test_diffusion_solve_without_host_checks_matches_checked_solve(mri):
    """check_every = 0 enqueues every iteration without synchronising: the launches
    after convergence do nothing, so the result and iteration count are the checked
    solve's; a solve cut short reports no convergence in cg_info."""
    import torch
    grid = mri.grid(24, 16, 8, 1e-4, (0.0, 0.0, 0.0), 1e-5, 2)
    n = 9
    b = torch.rand((24 * 16 * 8, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    ws = torch.empty(mri.mri_diffusion_workspace_size(grid, n), dtype=torch.uint8, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    x1 = b.clone()
    its = mri.mri_diffusion_solve(x1, b, grid, 1e-2, ws, tol=1e-13, max_iter=500, check_every=1, cg_info=info)
    assert info.tolist() == [1, its]
    x0 = b.clone()
    assert mri.mri_diffusion_solve(x0, b, grid, 1e-2, ws, tol=1e-13, max_iter=500, check_every=0, cg_info=info) == -1
    torch.cuda.synchronize()
    assert info.tolist() == [1, its]
    assert torch.equal(x0, x1)
    x2 = b.clone()
    mri.mri_diffusion_solve(x2, b, grid, 1e-2, ws, tol=1e-13, max_iter=3, check_every=0, cg_info=info)
    torch.cuda.synchronize()
    assert info.tolist() == [0, 3]


def test_imex1_step_captured_in_a_cuda_graph(mri, orc):
    """The IMEX step with cg_check_every = 0 recorded once in a CUDA graph and
    replayed for two steps, against two oracle steps."""
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    g = dict(w.grid, D=w.grid["D"] * 200)
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    m = orc.Mech(w.mech)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, w.H / 3, w.h, orc.opts(method=w.method, ramp=w.ramp))
    H = w.H / 2
    ref = y0
    for _ in range(2):
        ref, rst, _ = orc.imex1_step(m, ref, w.p, g, H, w.h, orc.opts(method=w.method))
        assert np.all(rst == 0)
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.tensor(y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    st = torch.zeros(y0.shape[0], dtype=torch.int32, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    ws = torch.empty(mri.mri_step_imex1_workspace_size(grid, w.mech.n), dtype=torch.uint8, device="cuda")
    opts = mri.mri_fast_opts_default(method=w.method, jac_policy=1)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    y_cap = y.clone()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=s):
        mri.mri_step_imex1(y_cap, p, grid, 0.0, H, w.h, gm, opts, ws, cg_tol=1e-14, cg_max_iter=200,
                           cg_check_every=0, cell_status=st, cg_info=info, stream=s)
    y_cap.copy_(y)
    torch.cuda.synchronize()
    iters = []
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        iters.append(info.tolist())
    assert all(c == 1 and 0 < k < 200 for c, k in iters), iters
    assert_parity(y_cap.cpu().numpy(), ref, what="IMEX1 two graph replays, box 8^3")


@pytest.mark.parametrize("name,cells", [("line64", None), ("box32", 8)])
def test_imex2_steps_match_oracle(mri, orc, name, cells):
    """Two second-order Strang-split IMEX steps (Crank-Nicolson half steps of the
    diffusion around the MRI3 step) against the oracle's.  Six fast stages of the hot
    box, each accepted at the Newton tolerance, with the state moved by the implicit
    half steps in between: both sides solve the stage equations to 1e-11 here, so
    that the comparison measures the implementations rather than where Newton
    stopped (at 1e-10 the two steps differ by 1.2e-10 on the box)."""
    import torch
    w = mechgen.workload(name, cells_per_side=cells)
    g = dict(w.grid, D=w.grid["D"] * 200)
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    m = orc.Mech(w.mech)
    y0, _, _ = m.stage_fast(w.y0, w.p, None, w.H / 3, w.h, orc.opts(method=w.method, ramp=w.ramp))
    rtol = 1e-11
    ref = y0
    for _ in range(2):
        ref, rst, _ = orc.imex2_step(m, ref, w.p, g, w.H, w.h, orc.opts(method=w.method, rtol=rtol))
        assert np.all(rst == 0)
    gm = mri.mri_mech_load(w.mech.to_blob())
    y = torch.tensor(y0, device="cuda")
    p = torch.tensor(w.p, device="cuda")
    st = torch.zeros(y0.shape[0], dtype=torch.int32, device="cuda")
    ws = torch.empty(mri.mri_step_imex2_workspace_size(grid, w.mech.n), dtype=torch.uint8, device="cuda")
    opts = mri.mri_fast_opts_default(method=w.method, jac_policy=1, newton_rtol=rtol)
    its = [mri.mri_step_imex2(y, p, grid, s * w.H, w.H, w.h, gm, opts, ws, cg_tol=1e-14, cell_status=st)
           for s in range(2)]
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0 and all(k > 0 for k in its)
    assert_parity(y.cpu().numpy(), ref, what=f"IMEX2 two steps {name}")


def test_imex2_step_in_a_cuda_graph_equals_the_direct_call(mri):
    """The second-order step with cg_check_every = 0 recorded in a CUDA graph and
    replayed gives bitwise the direct call's result (the kernels are deterministic)."""
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    g = dict(w.grid, D=w.grid["D"] * 200)
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    gm = mri.mri_mech_load(w.mech.to_blob())
    p = torch.tensor(w.p, device="cuda")
    y0 = torch.tensor(w.y0, device="cuda")
    mri.mri_stage_fast(y0, p, None, 0.0, w.H / 3, w.h, gm,
                       mri.mri_fast_opts_default(method=w.method, jac_policy=1, ramp=w.ramp))
    ws = torch.empty(mri.mri_step_imex2_workspace_size(grid, w.mech.n), dtype=torch.uint8, device="cuda")
    opts = mri.mri_fast_opts_default(method=w.method, jac_policy=1)
    direct = y0.clone()
    mri.mri_step_imex2(direct, p, grid, 0.0, w.H, w.h, gm, opts, ws, cg_tol=1e-13, cg_max_iter=40, cg_check_every=0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    y = y0.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        mri.mri_step_imex2(y, p, grid, 0.0, w.H, w.h, gm, opts, ws, cg_tol=1e-13, cg_max_iter=40, cg_check_every=0,
                           stream=s)
    y.copy_(y0)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, direct)


def test_imex2_cg_info_covers_both_half_steps(mri):
    """cg_info of the second-order step reports both Crank-Nicolson half steps: with no
    host checks and an iteration cap below what the first half step needs, it shows no
    convergence and the iterations of both; uncapped, it shows convergence and the
    same total as the host-checked step."""
    import torch
    w = mechgen.workload("box32", cells_per_side=8)
    g = dict(w.grid, D=w.grid["D"] * 200)
    grid = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], g["u"], g["D"], g["order"])
    gI = mri.grid(g["nx"], g["ny"], g["nz"], g["dx"], (0.0, 0.0, 0.0), g["D"], 2)
    n = w.mech.n
    gm = mri.mri_mech_load(w.mech.to_blob())
    p = torch.tensor(w.p, device="cuda")
    o = mri.mri_fast_opts_default(method=w.method, jac_policy=1, ramp=w.ramp)
    y0 = torch.tensor(w.y0, device="cuda")
    H = w.H / 2
    ws = torch.empty(mri.mri_step_imex2_workspace_size(grid, n), dtype=torch.uint8, device="cuda")
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    y = y0.clone()
    total = mri.mri_step_imex2(y, p, grid, 0.0, H, w.h, gm, o, ws, cg_tol=1e-13, cg_check_every=1)
    # the first half step alone through the public calls: (I - aL) x = (I + aL) y0, x from y0
    a = H / 4
    fI = torch.empty_like(y0)
    mri.mri_slow_rhs(y0, fI, gI)
    rhs = y0 + a * fI
    x = y0.clone()
    cws = torch.empty(mri.mri_diffusion_workspace_size(gI, n), dtype=torch.uint8, device="cuda")
    it1 = mri.mri_diffusion_solve(x, rhs, gI, a, cws, tol=1e-13, max_iter=1000, check_every=1)
    assert 2 <= it1 < total
    y = y0.clone()
    assert mri.mri_step_imex2(y, p, grid, 0.0, H, w.h, gm, o, ws, cg_tol=1e-13, cg_max_iter=1000,
                              cg_check_every=0, cg_info=info) == -1
    assert info.tolist() == [1, total]
    cap = it1 - 1
    y = y0.clone()
    info.fill_(7)
    mri.mri_step_imex2(y, p, grid, 0.0, H, w.h, gm, o, ws, cg_tol=1e-13, cg_max_iter=cap, cg_check_every=0,
                       cg_info=info)
    conv, its = info.tolist()
    assert conv == 0
    assert cap < its <= 2 * cap
