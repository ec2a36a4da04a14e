"""Accuracy of the kernels' own FP64 exponential and logarithm (table-driven,
after Tang 1989 and 1990) against libm on the host: at most 1 ulp (exp) and 2 ulp
(log, 1 ulp before the last rounding) on the ranges the rates use, and the library's results for the special
arguments each hands to the library function."""
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


def test_log_accuracy(mri):
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(200.0, 6000.0, 200000), 10.0 ** rng.uniform(-300, 300, 200000),
                        rng.uniform(0.99, 1.01, 100000), rng.uniform(1.0, 2.0, 100000),
                        [1.0, 2.0, 0.5, 1.0 + 2 ** -52, 1.0 - 2 ** -53, 1.5, 3.0, 1e300, 2.3e-308, 1000.0]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    mri.mri_probe_log(xd, yd)
    y = yd.cpu().numpy()
    ref = np.log(x)
    nz = ref != 0
    assert ulp_err(y[nz], ref[nz]).max() <= 2.0
    assert np.all(y[~nz] == 0.0)


def test_log_special_arguments(mri):
    import torch
    x = np.array([0.0, -0.0, -1.0, 1e-310, 4.9e-324, np.inf, -np.inf, np.nan])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    mri.mri_probe_log(xd, yd)
    y = yd.cpu().numpy()
    ref = torch.log(xd).cpu().numpy()
    np.testing.assert_array_equal(np.isnan(y), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(y[ok], ref[ok])


def test_exp_pair_accuracy(mri):
    """exp(x) and exp(-x) from one reduction, as the species factors are formed."""
    import torch
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-699, 699, 200000), rng.uniform(-50, 50, 100000), rng.uniform(-1e-6, 1e-6, 1000),
                        [0.0, 1.0, -1.0, 699.0, -699.0], [705.0, -705.0, 800.0, np.nan]])
    xd = torch.tensor(x, device="cuda")
    yd, zd = torch.empty_like(xd), torch.empty_like(xd)
    mri.mri_probe_exp_pair(xd, yd, zd)
    y, z = yd.cpu().numpy(), zd.cpu().numpy()
    body = np.abs(x) < 700
    assert ulp_err(y[body], np.exp(x[body])).max() <= 1.0
    assert ulp_err(z[body], np.exp(-x[body])).max() <= 1.0
    ref_y, ref_z = torch.exp(xd).cpu().numpy(), torch.exp(-xd).cpu().numpy()
    np.testing.assert_array_equal(y[~body], ref_y[~body])
    np.testing.assert_array_equal(z[~body], ref_z[~body])
