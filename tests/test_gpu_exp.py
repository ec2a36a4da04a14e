"""Accuracy of the kernels' own FP64 exponential (table-driven, after Tang 1989)
against libm on the host: at most 1 ulp on the ranges the rates use, and the
library exp's results (overflow, underflow, NaN) outside |x| < 700."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ulp_err(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_exp_accuracy(mri):
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-700, 700, 200000), rng.uniform(-1, 1, 100000), rng.uniform(-1e-8, 1e-8, 1000),
                        np.arange(-700, 701, 0.5), [0.0, -0.0, 699.999, -699.999, 1e-300, -1e-300]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    mri.mri_probe_exp(xd, yd)
    y = yd.cpu().numpy()
    ref = np.exp(x)
    assert ulp_err(y, ref).max() <= 1.0


def test_exp_special_arguments(mri):
    import torch
    x = np.array([710.0, 800.0, -750.0, -800.0, np.inf, -np.inf, np.nan, 705.0, -705.0])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    mri.mri_probe_exp(xd, yd)
    y = yd.cpu().numpy()
    ref = torch.exp(xd).cpu().numpy()
    np.testing.assert_array_equal(np.isnan(y), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(y[ok], ref[ok])
