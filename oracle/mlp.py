"""CPU oracle of the learned form's network -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the bench's CPU-baseline leg may import this
module; the product path never does.

A multilayer perceptron with SiLU hidden activations, written out in float64
numpy from the definitions:

    a_0 = x,  z_l = a_{l-1} W_l^T + b_l,  a_l = silu(z_l)  (hidden layers),
    y = z_L (linear output),  silu(z) = z / (1 + e^{-z}),

and its gradient by the chain rule for the loss  L = sum_{b,j} m_j (y_bj - t_bj)^2 / (2 B)
(a per-output weight m_j, mean over the batch B):

    dy = m (y - t) / B,  dz_L = dy,  dz_l = (dz_{l+1} W_{l+1}) * silu'(z_l),
    dW_l = dz_l^T a_{l-1},  db_l = sum_b dz_l,
    silu'(z) = s (1 + z (1 - s)),  s = 1 / (1 + e^{-z}).

``bf16=True`` rounds the weights and every GEMM input (x and the hidden
activations) to bfloat16 (round to nearest even) before it is multiplied, the
points at which the GPU kernels store bfloat16; all arithmetic stays float64.
The backward pass then rounds dz_l to bfloat16 where it enters a GEMM.
Parity pinned by central finite differences of the loss (tests).
"""
import numpy as np


def round_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    # NaN/inf pass through unchanged
    bad = ~np.isfinite(f)
    out[bad] = f[bad]
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, bf16=False):
    """params: list of (W [out, in], b [out]).  Returns (y, cache) with cache the
    per-layer (GEMM input, pre-activation)."""
    r = round_bf16 if bf16 else (lambda v: v)
    a = np.asarray(x, dtype=np.float64)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        ain = r(a)
        z = ain @ r(W).T + b
        cache.append((ain, z))
        a = silu(z) if l < L - 1 else z
    return a, cache


def loss(params, x, t, m, bf16=False):
    y, _ = forward(params, x, bf16)
    return float(np.sum(m * (y - t) ** 2) / (2.0 * x.shape[0]))


def backward(params, cache, y, t, m, bf16=False):
    """Gradients [(dW, db)] of ``loss`` for the forward pass that produced cache and y."""
    r = round_bf16 if bf16 else (lambda v: v)
    B = y.shape[0]
    dz = m * (y - t) / B
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        ain, z = cache[l]
        W, _ = params[l]
        if l < len(params) - 1:
            dz = dz * dsilu(z)
        dzr = r(dz)
        grads[l] = (dzr.T @ ain, dz.sum(axis=0))
        dz = dzr @ r(W)          # gradient with respect to this layer's input
    return grads


def adam_step(w, g, mom, vel, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of float64 arrays in place."""
    mom *= beta1
    mom += (1.0 - beta1) * g
    vel *= beta2
    vel += (1.0 - beta2) * g * g
    mhat = mom / (1.0 - beta1 ** step)
    vhat = vel / (1.0 - beta2 ** step)
    w -= lr * mhat / (np.sqrt(vhat) + eps)
