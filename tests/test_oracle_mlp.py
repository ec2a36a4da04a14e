"""Pins of the CPU oracle of the learned form's network (oracle/mlp.py): the
backward pass against central finite differences of the loss, bfloat16 rounding
against exactly representable cases, and the Adam update against its closed form
on the first step."""
import numpy as np

from oracle import mlp


def small_net(rng, sizes):
    return [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = small_net(rng, [7, 9, 8, 5])
    x = rng.standard_normal((6, 7))
    t = rng.standard_normal((6, 5))
    m = rng.uniform(0.5, 2.0, 5)
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t, m)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + eps
                lp = mlp.loss(params, x, t, m)
                arr[idx] = old - eps
                lm = mlp.loss(params, x, t, m)
                arr[idx] = old
                fd[idx] = (lp - lm) / (2 * eps)
            np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_silu_derivative_matches_finite_differences():
    z = np.linspace(-12, 12, 97)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-10)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.dsilu(0.0) - 0.5) < 1e-15


def test_bf16_rounding():
    # exactly representable values survive; halfway cases go to the even neighbour
    one = 1.0
    ulp = 2.0 ** -7                        # bfloat16 spacing just above 1
    vals = np.array([one, -2.5, 0.0, one + ulp, one + ulp / 2, one + 3 * ulp / 2, one + ulp / 2 + 2.0 ** -20,
                     3.0e38, 1e-40])
    got = mlp.round_bf16(vals)
    np.testing.assert_array_equal(got[:4], [1.0, -2.5, 0.0, one + ulp])
    assert got[4] == 1.0                   # tie -> even (mantissa ...0)
    assert got[5] == one + 2 * ulp         # tie -> even (mantissa ...0)
    assert got[6] == one + ulp             # above the tie -> up
    assert np.isfinite(got[7]) and abs(got[7] / 3.0e38 - 1) <= 2.0 ** -8
    assert 0.0 <= got[8] <= 2e-40            # float32 subnormals round within the subnormal range
    rel = np.abs(mlp.round_bf16(np.linspace(1, 2, 1001)) / np.linspace(1, 2, 1001) - 1)
    assert rel.max() <= 2.0 ** -8 + 1e-15


def test_bf16_forward_stays_close_to_exact():
    rng = np.random.default_rng(1)
    params = small_net(rng, [16, 32, 32, 4])
    x = rng.standard_normal((64, 16))
    y64, _ = mlp.forward(params, x)
    y16, _ = mlp.forward(params, x, bf16=True)
    assert np.abs(y16 - y64).max() <= 0.05 * np.abs(y64).max()


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    w = rng.standard_normal(10)
    g = rng.standard_normal(10)
    mom, vel = np.zeros(10), np.zeros(10)
    w0 = w.copy()
    mlp.adam_step(w, g, mom, vel, 1, lr=1e-2, eps=1e-8)
    # first step: mhat = g, vhat = g^2, so the update is lr g / (|g| + eps)
    np.testing.assert_allclose(w, w0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14)
