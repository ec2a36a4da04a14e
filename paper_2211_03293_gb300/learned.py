"""Learned form of the fast solve: data, training and use of the network that
predicts a stage's substep-end states as the Newton start of the fast solve.

Every computation runs in the library's kernels (include/mri_mlp.h, mri.h):
the plain solver produces the training data, the data kernels standardise and
shuffle it on the device, the tensor-core network kernels train and evaluate the
model, and mri_stage_fast_guided solves the stage from the predicted states --
every stage value is still accepted only by the FP64 Newton residual test, with a
restart from the plain start wherever Newton does not converge.  This module only
sequences those calls; the host draws the shuffles' permutations (seeded) and
reads back the step network's two normalisation constants.
"""
from __future__ import annotations

import math

import numpy as np

from . import (Mlp, mri_fast_opts, mri_learned_features, mri_learned_guess, mri_learned_moments,
               mri_learned_standardise, mri_learned_step_exp, mri_learned_step_targets, mri_learned_targets,
               mri_mlp_adam, mri_mlp_forward, mri_mlp_grad, mri_stage_fast)


def _pad16(v):
    return (v + 15) // 16 * 16


def n_substeps(Hstage, h):
    return max(1, math.ceil(Hstage / h * (1.0 - 1e-12)))


def stage_substep_states(y, p, phi, Hstage, h, mech, opts, stream=None):
    """Integrate one fast stage a substep at a time with the plain solver and return
    (states at the substep ends [ncell][G][n], G).  y is advanced in place to the
    stage output.  The forcing must be constant over the stage (K <= 1, the MIS
    form's case), so that each single-substep call sees the same forcing."""
    import torch
    if phi is not None and phi.shape[1] > 1:
        raise ValueError("substep-wise data needs a constant stage forcing (K <= 1)")
    G = n_substeps(Hstage, h)
    hh = Hstage / G
    seq = torch.empty((y.shape[0], G, y.shape[1]), dtype=torch.float64, device=y.device)
    for g in range(G):
        o = mri_fast_opts.from_buffer_copy(opts)
        if g > 0:
            o.ramp = 0
        mri_stage_fast(y, p, phi, g * hh, hh, hh, mech, o, stream=stream)
        seq[:, g, :].copy_(y)
    return seq, G


class LearnedStart:
    """Network (inputs 2n + 2 features, 3 x 256 SiLU, outputs g_max n substep-end
    increments) with the standardisation of its inputs and outputs."""

    def __init__(self, n, g_max, hidden=256, layers=3, batch=4096, seed=0, infer_batch=None):
        import torch
        self.n, self.g_max, self.batch = n, g_max, batch
        self.infer_batch = infer_batch or batch
        self.n_in = _pad16(2 * n + 2)
        self.n_out = _pad16(g_max * n)
        self.dims = [self.n_in] + [hidden] * layers + [self.n_out]
        rng = np.random.default_rng(seed)
        params = []
        for i, o in zip(self.dims[:-1], self.dims[1:]):
            params.append(rng.standard_normal((o, i)).astype(np.float32).ravel() * np.float32(np.sqrt(1.0 / i)))
            params.append(np.zeros(o, dtype=np.float32))
        self.net = Mlp(self.dims, max(batch, self.infer_batch), np.concatenate(params))
        dev = torch.device("cuda")
        f32 = dict(dtype=torch.float32, device=dev)
        self.fmean = torch.zeros(self.n_in, **f32)
        self.finv = torch.ones(self.n_in, **f32)
        self.tmean = torch.zeros(self.n_out, **f32)
        self.tstd = torch.ones(self.n_out, **f32)
        self.w_out = torch.zeros(self.n_out, **f32)
        self.records = []
        self.step = 0

    # ------------------------------------------------------------------ data
    def add(self, y_in, p, phi, Hstage, y_seq):
        """Keep one stage's example: raw features and raw targets (device float32)."""
        import torch
        ncell, n = y_in.shape
        G = y_seq.shape[1]
        if G > self.g_max:
            raise ValueError("more substeps than the network predicts")
        # substeps beyond G repeat the stage output, so every output column is defined
        full = torch.empty((ncell, self.g_max, n), dtype=torch.float64, device=y_in.device)
        full[:, :G].copy_(y_seq)
        full[:, G:].copy_(y_seq[:, G - 1:G].expand(ncell, self.g_max - G, n))
        x = torch.empty((ncell, self.n_in), dtype=torch.float32, device=y_in.device)
        zero_in = torch.zeros(self.n_in, dtype=torch.float32, device=y_in.device)
        one_in = torch.ones(self.n_in, dtype=torch.float32, device=y_in.device)
        mri_learned_features(y_in, p, phi, Hstage, zero_in, one_in, x)
        t = torch.empty((ncell, self.n_out), dtype=torch.float32, device=y_in.device)
        zero_out = torch.zeros(self.n_out, dtype=torch.float32, device=y_in.device)
        one_out = torch.ones(self.n_out, dtype=torch.float32, device=y_in.device)
        mri_learned_targets(y_in, full, zero_out, one_out, t)
        self.records.append((x, t))

    def _standardise(self):
        """Device standardisation constants of the collected examples; returns the raw
        feature and target matrices (device float32)."""
        import torch
        X = torch.cat([r[0] for r in self.records])
        T = torch.cat([r[1] for r in self.records])
        nf, used_out = 2 * self.n + 2, self.g_max * self.n
        fm, finv, _ = mri_learned_moments(X, nf, 1e-12)
        tm, tinv, ts = mri_learned_moments(T, used_out, 1e-30)
        dev = X.device
        f32 = dict(dtype=torch.float32, device=dev)
        self.fmean, self.finv = torch.zeros(self.n_in, **f32), torch.ones(self.n_in, **f32)
        self.fmean[:nf].copy_(fm)
        self.finv[:nf].copy_(finv)
        self.tmean, self.tstd = torch.zeros(self.n_out, **f32), torch.ones(self.n_out, **f32)
        self.tmean[:used_out].copy_(tm)
        self.tstd[:used_out].copy_(ts)
        self._tinv = torch.ones(self.n_out, **f32)
        self._tinv[:used_out].copy_(tinv)
        self.w_out = torch.zeros(self.n_out, **f32)
        self.w_out[:used_out] = 1.0
        return X, T

    # ------------------------------------------------------------------ training
    def fit(self, epochs=100, lr=1e-3, seed=0, stream=None, log=None):
        """Adam on minibatches of the collected examples, standardised and shuffled (once,
        with a seeded permutation) on the device.  Returns the loss history (one value per
        epoch, the last minibatch's)."""
        import torch
        X, T = self._standardise()
        N = X.shape[0]
        nb = N // self.batch
        if nb < 1:
            raise ValueError("fewer examples than one minibatch")
        dev = X.device
        perm = torch.tensor(np.random.default_rng(seed).permutation(N)[:nb * self.batch].astype(np.int32), device=dev)
        Xn = torch.empty((nb * self.batch, self.n_in), dtype=torch.float32, device=dev)
        Tn = torch.empty((nb * self.batch, self.n_out), dtype=torch.float32, device=dev)
        mri_learned_standardise(X, perm, 2 * self.n + 2, self.fmean, self.finv, Xn, stream=stream)
        mri_learned_standardise(T, perm, self.g_max * self.n, self.tmean, self._tinv, Tn, stream=stream)
        Xb = Xn.view(nb, self.batch, -1)
        Tb = Tn.view(nb, self.batch, -1)
        y = torch.empty((self.batch, self.n_out), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        hist = []
        for ep in range(epochs):
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))    # cosine decay
            for b in range(nb):
                mri_mlp_grad(self.net, Xb[b], Tb[b], self.w_out, y, loss, stream=stream)
                self.step += 1
                mri_mlp_adam(self.net, rate, self.step, stream=stream)
            hist.append(float(loss.item()))
            if log:
                log(ep, hist[-1])
        return hist

    # ------------------------------------------------------------------ use
    def guess(self, y_in, p, phi, Hstage, h, stream=None):
        """Predicted substep-end states [ncell][G][n] for a stage of length Hstage."""
        import torch
        ncell = y_in.shape[0]
        G = n_substeps(Hstage, h)
        dev = y_in.device
        out = torch.empty((ncell, G, self.n), dtype=torch.float64, device=dev)
        chunk = min(ncell, self.infer_batch)
        if getattr(self, "_xbuf", None) is None or self._xbuf.shape[0] < chunk:
            self._xbuf = torch.empty((chunk, self.n_in), dtype=torch.float32, device=dev)
            self._ybuf = torch.empty((chunk, self.n_out), dtype=torch.float32, device=dev)
        x, yh = self._xbuf, self._ybuf
        for c0 in range(0, ncell, chunk):
            c1 = min(ncell, c0 + chunk)
            m = c1 - c0
            ph = None if phi is None else phi[c0:c1]
            mri_learned_features(y_in[c0:c1], p[c0:c1], ph, Hstage, self.fmean, self.finv, x[:m], stream=stream)
            mri_mlp_forward(self.net, x[:m], yh[:m], stream=stream)
            mri_learned_guess(y_in[c0:c1], yh[:m], G, self.tmean, self.tstd, out[c0:c1], stream=stream)
        return out


class LearnedSteps:
    """Substep-size predictor: a network with the same inputs (2n + 2 features, 3 x 256
    SiLU) and one output, the log2 of the adaptive controller's mean accepted step
    relative to the uniform substep, k = log2(n_sub / accepted steps), per cell and
    stage.  Rounded and clamped it is the first-step exponent of an adaptive stage
    (mri_stage_fast_guided's step_exp), so that cells far from the uniform step size
    start near their own."""

    def __init__(self, n, hidden=256, layers=3, batch=4096, seed=1):
        import torch
        self.n, self.batch = n, batch
        self.n_in = _pad16(2 * n + 2)
        self.n_out = 16
        self.dims = [self.n_in] + [hidden] * layers + [self.n_out]
        rng = np.random.default_rng(seed)
        params = []
        for i, o in zip(self.dims[:-1], self.dims[1:]):
            params.append(rng.standard_normal((o, i)).astype(np.float32).ravel() * np.float32(np.sqrt(1.0 / i)))
            params.append(np.zeros(o, dtype=np.float32))
        self.net = Mlp(self.dims, batch, np.concatenate(params))
        dev = torch.device("cuda")
        self.fmean = torch.zeros(self.n_in, dtype=torch.float32, device=dev)
        self.finv = torch.ones(self.n_in, dtype=torch.float32, device=dev)
        self.kmean, self.kstd = 0.0, 1.0
        w = np.zeros(self.n_out, dtype=np.float32)
        w[0] = 1.0
        self.w_out = torch.tensor(w, device=dev)
        self.records = []
        self.step = 0

    def add(self, y_in, p, phi, Hstage, h, accepted):
        """One stage's examples: the stage inputs and the accepted step counts of an
        adaptive solve of it (int32, device or host: cell_stats[:, 0] or a whole
        cell_stats [ncell][4] tensor)."""
        import torch
        ncell = y_in.shape[0]
        dev = y_in.device
        x = torch.empty((ncell, self.n_in), dtype=torch.float32, device=dev)
        zero = torch.zeros(self.n_in, dtype=torch.float32, device=dev)
        one = torch.ones(self.n_in, dtype=torch.float32, device=dev)
        mri_learned_features(y_in, p, phi, Hstage, zero, one, x)
        if not torch.is_tensor(accepted):
            accepted = torch.tensor(np.asarray(accepted), dtype=torch.int32, device=dev)
        stride = 4 if accepted.dim() == 2 else 1
        acc = accepted.to(device=dev, dtype=torch.int32).contiguous()
        k = torch.empty((ncell, 1), dtype=torch.float32, device=dev)
        mri_learned_step_targets(acc, n_substeps(Hstage, h), k, stride=stride)
        self.records.append((x, k))

    def fit(self, epochs=100, lr=1e-3, seed=0, stream=None):
        """Adam on the collected examples, standardised and shuffled on the device."""
        import torch
        X = torch.cat([r[0] for r in self.records])
        K = torch.cat([r[1] for r in self.records])
        nf = 2 * self.n + 2
        dev = X.device
        fm, finv, _ = mri_learned_moments(X, nf, 1e-12)
        km, kinv, ks = mri_learned_moments(K, 1, 1e-6)
        self.fmean = torch.zeros(self.n_in, dtype=torch.float32, device=dev)
        self.finv = torch.ones(self.n_in, dtype=torch.float32, device=dev)
        self.fmean[:nf].copy_(fm)
        self.finv[:nf].copy_(finv)
        self.kmean, self.kstd = float(km.item()), float(ks.item())
        N = X.shape[0]
        nb = N // self.batch
        if nb < 1:
            raise ValueError("fewer examples than one minibatch")
        perm = torch.tensor(np.random.default_rng(seed).permutation(N)[:nb * self.batch].astype(np.int32), device=dev)
        Xd = torch.empty((nb * self.batch, self.n_in), dtype=torch.float32, device=dev)
        Td = torch.empty((nb * self.batch, self.n_out), dtype=torch.float32, device=dev)
        mri_learned_standardise(X, perm, nf, self.fmean, self.finv, Xd, stream=stream)
        mri_learned_standardise(K, perm, 1, km, kinv, Td, stream=stream)
        Xd = Xd.view(nb, self.batch, -1)
        Td = Td.view(nb, self.batch, -1)
        y = torch.empty((self.batch, self.n_out), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        hist = []
        for ep in range(epochs):
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))
            for bi in range(nb):
                mri_mlp_grad(self.net, Xd[bi], Td[bi], self.w_out, y, loss, stream=stream)
                self.step += 1
                mri_mlp_adam(self.net, rate, self.step, stream=stream)
            hist.append(float(loss.item()))
        return hist

    def step_exp(self, y_in, p, phi, Hstage, kmin=-20, kmax=10, stream=None):
        """Predicted first-step exponents (int8 [ncell], device)."""
        import torch
        ncell = y_in.shape[0]
        dev = y_in.device
        out = torch.empty(ncell, dtype=torch.int8, device=dev)
        x = torch.empty((min(ncell, self.batch), self.n_in), dtype=torch.float32, device=dev)
        yh = torch.empty((min(ncell, self.batch), self.n_out), dtype=torch.float32, device=dev)
        for c0 in range(0, ncell, self.batch):
            c1 = min(ncell, c0 + self.batch)
            m = c1 - c0
            ph = None if phi is None else phi[c0:c1]
            mri_learned_features(y_in[c0:c1], p[c0:c1], ph, Hstage, self.fmean, self.finv, x[:m], stream=stream)
            mri_mlp_forward(self.net, x[:m], yh[:m], stream=stream)
            mri_learned_step_exp(yh[:m], 0, self.kmean, self.kstd, out[c0:c1], kmin, kmax, stream=stream)
        return out
