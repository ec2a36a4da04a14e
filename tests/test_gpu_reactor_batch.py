"""A batch of 4096 independent constant-pressure 0-D reactors on three mechanisms
(9 species / 21 reactions, 40 / 170, 80 / 350) advanced in one launch of
mri_stage_fast_batch: parity with the CPU oracle on sampled reactors of every
group, and bitwise agreement with one mri_stage_fast launch per group."""
import numpy as np
import pytest

import mechgen
from _parity import assert_parity

pytestmark = pytest.mark.gpu


def device_groups(mri, batch):
    import torch
    out = []
    for mech, y, p in batch.groups:
        nc = y.shape[0]
        out.append(dict(mech=mri.mri_mech_load(mech.to_blob()), y=torch.tensor(y, device="cuda"),
                        p=torch.tensor(p, device="cuda"),
                        cell_status=torch.full((nc,), -9, dtype=torch.int32, device="cuda"),
                        cell_stats=torch.zeros((nc, 4), dtype=torch.int32, device="cuda")))
    return out


def opts(mri, batch, prec):
    return mri.mri_fast_opts_default(method=batch.method, newton_rtol=batch.newton_rtol, ramp=batch.ramp,
                                     jac_policy=mri.MRI_JAC_LAZY, precision=prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_batch_equals_one_launch_per_group(mri, prec):
    import torch
    batch = mechgen.reactor_batch()
    o = opts(mri, batch, prec)
    mixed = device_groups(mri, batch)
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    mri.mri_stage_fast_batch(mixed, 0.0, batch.Hstage, batch.h, o, n_failed=nf)
    single = device_groups(mri, batch)
    for g in single:
        mri.mri_stage_fast(g["y"], g["p"], None, 0.0, batch.Hstage, batch.h, g["mech"], o,
                           cell_status=g["cell_status"], cell_stats=g["cell_stats"])
    torch.cuda.synchronize()
    assert int(nf.item()) == 0
    for a, b in zip(mixed, single):
        for k in ("y", "cell_status", "cell_stats"):
            np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy())
        assert np.all(a["cell_status"].cpu().numpy() == 0)


def test_mixed_batch_parity_sampled(mri, orc):
    import torch
    batch = mechgen.reactor_batch()
    mixed = device_groups(mri, batch)
    mri.mri_stage_fast_batch(mixed, 0.0, batch.Hstage, batch.h, opts(mri, batch, 0))
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for (mech, y, p), g in zip(batch.groups, mixed):
        idx = np.sort(rng.choice(y.shape[0], 24, replace=False))
        ref, rst, rss = orc.Mech(mech).stage_fast(y[idx], p[idx], None, batch.Hstage, batch.h,
                                                  orc.opts(method=batch.method, rtol=batch.newton_rtol,
                                                           ramp=batch.ramp))
        assert np.all(rst == 0)
        got = g["y"].cpu().numpy()[idx]
        assert_parity(got, ref, what=f"{mech.n_species}-species reactors")
        ss = g["cell_stats"].cpu().numpy()[idx]
        assert np.all(ss[:, 0] == rss[:, 0])          # same substep count


def test_mixed_batch_with_empty_group_and_forcing(mri):
    """Groups may be empty; a group may carry forcing coefficients (K > 0) while the
    others have none."""
    import torch
    batch = mechgen.reactor_batch(n_reactors=300)
    groups = device_groups(mri, batch)
    groups[0]["y"] = groups[0]["y"][:0]
    groups[0]["p"] = groups[0]["p"][:0]
    groups[0]["cell_status"] = groups[0]["cell_status"][:0]
    groups[0]["cell_stats"] = groups[0]["cell_stats"][:0]
    mech1, y1, p1 = batch.groups[1]
    phi = mechgen.random_forcing(4, y1.shape[0], mech1.n, 2)
    groups[1]["phi"] = torch.tensor(phi, device="cuda")
    o = opts(mri, batch, 0)
    mri.mri_stage_fast_batch(groups, 0.0, batch.Hstage, batch.h, o)
    ref = device_groups(mri, batch)
    mri.mri_stage_fast(ref[1]["y"], ref[1]["p"], groups[1]["phi"], 0.0, batch.Hstage, batch.h, ref[1]["mech"], o)
    mri.mri_stage_fast(ref[2]["y"], ref[2]["p"], None, 0.0, batch.Hstage, batch.h, ref[2]["mech"], o)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(groups[1]["y"].cpu().numpy(), ref[1]["y"].cpu().numpy())
    np.testing.assert_array_equal(groups[2]["y"].cpu().numpy(), ref[2]["y"].cpu().numpy())
