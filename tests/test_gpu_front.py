"""Full-size workloads of the batched and precision forms.

* The 128^3 box with a planar flame front (2.1M cells): the per-cell Newton and
  Jacobian work varies several-fold between the cold gas, the front and the hot
  products, which is what the persistent kernel's work queue balances.  One fast
  stage (with the start-up ramp) of the whole box, compared with the oracle on
  sampled cells, and the spread of the per-cell work reported by the kernel.
* The 64^3 box in the mixed-precision form (FP32 Newton matrix and LU, FP64
  rates and residual): sampled cells of a full-size stage against the FP64 oracle,
  with the maximum and RMS relative error per field."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def full_stage(mri, w, phi, opts):
    import torch
    gm = mri.mri_mech_load(w.mech.to_blob())
    yd = torch.tensor(w.y0, device="cuda")
    pd = torch.tensor(w.p, device="cuda")
    ph = torch.tensor(phi, device="cuda")
    st = torch.zeros(w.y0.shape[0], dtype=torch.int32, device="cuda")
    ss = torch.zeros((w.y0.shape[0], 4), dtype=torch.int32, device="cuda")
    mri.mri_stage_fast(yd, pd, ph, 0.0, w.H / 3, w.h, gm, opts, cell_status=st, cell_stats=ss)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), ss.cpu().numpy()


def test_front128_full_stage_sampled_parity_and_uneven_work(mri, orc):
    w = mechgen.workload("front128")
    phi = mechgen.random_forcing(9, w.y0.shape[0], w.mech.n, 1)
    for prec in (0, 1):
        opts = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=mri.MRI_JAC_LAZY, precision=prec)
        got, st, ss = full_stage(mri, w, phi, opts)
        assert int((st != 0).sum()) == 0
        rng = np.random.default_rng(1)
        idx = np.sort(rng.choice(w.y0.shape[0], 32, replace=False))
        ref, rst, _ = orc.Mech(w.mech).stage_fast(w.y0[idx], w.p[idx], phi[idx], w.H / 3, w.h,
                                                  orc.opts(method=3, ramp=w.ramp))
        assert np.all(rst == 0)
        assert_parity(got[idx], ref, what=f"front 128^3 (form {prec})")
        # uneven work: Newton iterations and Jacobians per cell across the front
        newton, njac = ss[:, 1], ss[:, 2]
        print(f"form {prec}: Newton per cell min {newton.min()} median {np.median(newton)} max {newton.max()}; "
              f"Jacobians min {njac.min()} max {njac.max()}")
        assert newton.max() >= 2 * newton.min()


def test_box64_mixed_precision_full_stage_per_field_error(mri, orc):
    w = mechgen.workload("box64")
    phi = mechgen.random_forcing(10, w.y0.shape[0], w.mech.n, 1)
    opts = mri.mri_fast_opts_default(method=3, ramp=w.ramp, jac_policy=mri.MRI_JAC_LAZY,
                                     precision=mri.MRI_PREC_FP32_LU)
    got, st, _ = full_stage(mri, w, phi, opts)
    assert int((st != 0).sum()) == 0
    idx = np.sort(np.random.default_rng(2).choice(w.y0.shape[0], 48, replace=False))
    ref, rst, _ = orc.Mech(w.mech).stage_fast(w.y0[idx], w.p[idx], phi[idx], w.H / 3, w.h,
                                              orc.opts(method=3, ramp=w.ramp))
    assert np.all(rst == 0)
    g = got[idx]
    big = ref[:, :-1] > 1e-10
    ry = np.abs(g[:, :-1] - ref[:, :-1])[big] / ref[:, :-1][big]
    rt = np.abs(g[:, -1] - ref[:, -1]) / ref[:, -1]
    print(f"64^3 mixed form vs FP64 oracle: Y max {ry.max():.2e} rms {np.sqrt(np.mean(ry ** 2)):.2e}; "
          f"T max {rt.max():.2e} rms {np.sqrt(np.mean(rt ** 2)):.2e}")
    assert_parity(g, ref, what="64^3 mixed form")
