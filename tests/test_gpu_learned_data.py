"""The learned form's data kernels on the device against numpy: column moments of a
training matrix, the standardised and shuffled copy of its rows, and the targets of
the substep-size network from accepted step counts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_moments_and_standardise_match_numpy(mri):
    import torch
    rng = np.random.default_rng(7)
    rows, ld, used = 100003, 112, 98
    X = (rng.standard_normal((rows, ld)) * rng.uniform(0.01, 30, ld) + rng.uniform(-5, 5, ld)).astype(np.float32)
    X[:, 3] = 2.5                                                    # a constant column
    Xd = torch.tensor(X, device="cuda")
    mean, inv, sd = mri.mri_learned_moments(Xd, used, 1e-12)
    X64 = X[:, :used].astype(np.float64)
    m_ref, s_ref = X64.mean(0), X64.std(0)
    s_ref[s_ref < 1e-12] = 1.0
    np.testing.assert_allclose(mean.cpu().numpy(), m_ref, rtol=1e-6, atol=1e-6 * np.abs(m_ref).max())
    np.testing.assert_allclose(sd.cpu().numpy(), s_ref, rtol=1e-5)
    np.testing.assert_allclose(inv.cpu().numpy(), 1.0 / s_ref, rtol=1e-5)
    assert sd.cpu().numpy()[3] == 1.0
    perm = rng.permutation(rows)[:65536].astype(np.int32)
    out = torch.full((65536, 128), np.nan, dtype=torch.float32, device="cuda")
    mri.mri_learned_standardise(Xd, torch.tensor(perm, device="cuda"), used, mean, inv, out)
    got = out.cpu().numpy()
    ref = (X[perm, :used] - mean.cpu().numpy()) * inv.cpu().numpy()
    np.testing.assert_allclose(got[:, :used], ref, rtol=1e-6, atol=1e-6)
    assert np.all(got[:, used:] == 0.0)


def test_step_targets_match_numpy(mri):
    import torch
    rng = np.random.default_rng(8)
    acc = rng.integers(0, 3000, size=(5000, 4)).astype(np.int32)
    k = torch.empty(5000, dtype=torch.float32, device="cuda")
    mri.mri_learned_step_targets(torch.tensor(acc, device="cuda"), 12, k, stride=4)
    ref = np.log2(12.0 / np.maximum(acc[:, 0], 1)).astype(np.float32)
    np.testing.assert_array_equal(k.cpu().numpy(), ref)
