"""The learned form's network on the GPU: the tensor-core GEMM against numpy on
bfloat16-rounded operands, forward pass and parameter gradients against the CPU
oracle (oracle/mlp.py, float64 with the same bfloat16 rounding points) element by
element against each element's magnitude scale, and Adam training driving the loss
down."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def bf16_tensor(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 48, 96), (1000, 256, 256), (77, 128, 8), (5, 32, 200)])
def test_gemm_bf16_matches_numpy(mri, M, N, K):
    import torch
    rng = np.random.default_rng(M * 7 + N + K)
    A = omlp.round_bf16(rng.standard_normal((M, K)))
    B = omlp.round_bf16(rng.standard_normal((N, K)))
    C = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    mri.mri_gemm_bf16(bf16_tensor(A), bf16_tensor(B), C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-30), np.max(np.abs(got - ref) / scale)


def make_params(rng, dims):
    return [(rng.standard_normal((o, i)) * np.sqrt(2.0 / i), 0.1 * rng.standard_normal(o))
            for i, o in zip(dims[:-1], dims[1:])]


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def unpack(flat, dims):
    out, o = [], 0
    for i, n in zip(dims[:-1], dims[1:]):
        W = flat[o:o + i * n].reshape(n, i); o += i * n
        b = flat[o:o + n]; o += n
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


DIMS = [96, 256, 256, 256, 48]

# Elementwise comparison of the GPU network with the float64 oracle.  Each output
# element of a layer is a sum of products; its magnitude scale is the sum of the
# products' magnitudes (|a| |W|^T for a forward pre-activation, |dz|^T |a| for a weight
# gradient).  The GPU multiplies bfloat16 operands exactly and accumulates in FP32,
# which keeps a layer within about 1e-6 of that scale; where an activation lies within
# that distance of a bfloat16 rounding boundary, the two sides round it to neighbouring
# bfloat16 values, and such flips carry a difference of one bfloat16 step (2^-8
# relative) of one term into the next layer.  Every element must therefore stay within
# 1e-2 of its scale (several flips at once; an FP32 emulation of the GPU's arithmetic
# stays below 1e-3), and 99 per cent of the elements within 1e-3; a wrong term, row
# or column exceeds the first.
MAX_OF_SCALE = 1e-2
P99_OF_SCALE = 1e-3


def assert_elementwise(got, ref, scale, what):
    r = np.abs(got - ref) / np.maximum(scale, 1e-300)
    i = np.unravel_index(np.argmax(r), r.shape)
    assert r.max() <= MAX_OF_SCALE, f"{what}: element {i} off by {r[i]:.3e} of its scale"
    assert np.percentile(r, 99) <= P99_OF_SCALE, f"{what}: 99th percentile {np.percentile(r, 99):.3e}"


def layer_scales(params, cache, y, t, m):
    """Magnitude scales of the output and of every layer's weight and bias gradient,
    from the oracle's own pass."""
    B = y.shape[0]
    ain, _ = cache[-1]
    W, b = params[-1]
    out_scale = np.abs(ain) @ np.abs(omlp.round_bf16(W)).T + np.abs(b)
    dz = m * (y - t) / B
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        ain, z = cache[l]
        W, _ = params[l]
        if l < len(params) - 1:
            dz = dz * omlp.dsilu(z)
        dzr = omlp.round_bf16(dz)
        grads[l] = (np.abs(dzr).T @ np.abs(ain), np.abs(dz).sum(axis=0))
        dz = dzr @ omlp.round_bf16(W)
    return out_scale, grads


def test_forward_matches_oracle(mri):
    import torch
    rng = np.random.default_rng(1)
    params = make_params(rng, DIMS)
    flat = pack(params)
    net = mri.mri_mlp_create(DIMS, 1000, flat)
    params = unpack(flat, DIMS)          # the float32 values the GPU holds
    x = rng.standard_normal((999, DIMS[0]))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.zeros((999, DIMS[-1]), dtype=torch.float32, device="cuda")
    mri.mri_mlp_forward(net, xd, yd)
    torch.cuda.synchronize()
    assert mri.mri_mlp_status(net) == 0
    x64 = x.astype(np.float32).astype(np.float64)
    ref, cache = omlp.forward(params, x64, bf16=True)
    scale, _ = layer_scales(params, cache, ref, ref, np.ones(DIMS[-1]))
    assert_elementwise(yd.cpu().numpy().astype(np.float64), ref, scale, "forward output")


def test_gradients_match_oracle(mri):
    import torch
    rng = np.random.default_rng(2)
    params = make_params(rng, DIMS)
    flat = pack(params)
    B = 300
    net = mri.mri_mlp_create(DIMS, B, flat)
    params = unpack(flat, DIMS)
    x = rng.standard_normal((B, DIMS[0])).astype(np.float32)
    t = rng.standard_normal((B, DIMS[-1])).astype(np.float32)
    m = rng.uniform(0.5, 2.0, DIMS[-1]).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")
    y = torch.zeros((B, DIMS[-1]), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    mri.mri_mlp_grad(net, dev(x), dev(t), dev(m), y, loss)
    mri.mri_mlp_grad_copy(net, g)
    torch.cuda.synchronize()
    assert mri.mri_mlp_status(net) == 0
    yr, cache = omlp.forward(params, x.astype(np.float64), bf16=True)
    ref = omlp.backward(params, cache, yr, t.astype(np.float64), m.astype(np.float64), bf16=True)
    Lr = np.sum(m * (yr - t) ** 2) / (2 * B)
    assert abs(float(loss.item()) - Lr) <= 5e-3 * Lr
    got = unpack(g.cpu().numpy(), DIMS)
    _, scales = layer_scales(params, cache, yr, t.astype(np.float64), m.astype(np.float64))
    for l, ((gW, gb), (rW, rb), (sW, sb)) in enumerate(zip(got, ref, scales)):
        assert_elementwise(gW, rW, sW, f"layer {l} weight gradient")
        assert_elementwise(gb, rb, sb, f"layer {l} bias gradient")


def test_adam_training_reduces_the_loss(mri):
    """Fit a smooth map R^96 -> R^48 (a fixed random tanh layer) from 4096 samples."""
    import torch
    rng = np.random.default_rng(3)
    params = make_params(rng, DIMS)
    B = 4096
    net = mri.mri_mlp_create(DIMS, B, pack(params))
    x = rng.standard_normal((B, DIMS[0])).astype(np.float32)
    Wt = rng.standard_normal((DIMS[-1], DIMS[0])) / np.sqrt(DIMS[0])
    t = np.tanh(x @ Wt.T).astype(np.float32)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    m = torch.ones(DIMS[-1], dtype=torch.float32, device="cuda")
    y = torch.zeros((B, DIMS[-1]), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for step in range(1, 301):
        mri.mri_mlp_grad(net, xd, td, m, y, loss)
        mri.mri_mlp_adam(net, 1e-3, step)
        if step in (1, 300):
            torch.cuda.synchronize()
            hist.append(float(loss.item()))
    assert mri.mri_mlp_status(net) == 0
    assert hist[1] < 0.1 * hist[0], hist
