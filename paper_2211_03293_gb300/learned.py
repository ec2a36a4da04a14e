"""Learned form of the fast solve: data, training and use of the network that
predicts a stage's substep-end states as the Newton start of the fast solve.

Every computation runs in the library's kernels (include/mri_mlp.h, mri.h):
the plain solver produces the training data, the tensor-core network kernels
train and evaluate the model, and mri_stage_fast_guided solves the stage from
the predicted states -- every stage value is still accepted only by the FP64
Newton residual test, with a restart from the plain start wherever Newton does
not converge.  This module only sequences those calls and keeps the
normalisation constants (host arithmetic on data already produced).
"""
from __future__ import annotations

import math

import numpy as np

from . import (Mlp, mri_fast_opts, mri_learned_features, mri_learned_guess, mri_learned_step_exp,
               mri_learned_targets, mri_mlp_adam, mri_mlp_forward, mri_mlp_grad, mri_stage_fast)


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
        import torch
        X = torch.cat([r[0] for r in self.records]).cpu().numpy().astype(np.float64)
        T = torch.cat([r[1] for r in self.records]).cpu().numpy().astype(np.float64)
        fm, fs = X.mean(0), X.std(0)
        tm, ts = T.mean(0), T.std(0)
        used_out = self.g_max * self.n
        fs[fs < 1e-12] = 1.0
        ts[ts < 1e-30] = 1.0
        dev = self.fmean.device
        self.fmean = torch.tensor(fm, dtype=torch.float32, device=dev)
        self.finv = torch.tensor(1.0 / fs, dtype=torch.float32, device=dev)
        self.tmean = torch.tensor(tm, dtype=torch.float32, device=dev)
        self.tstd = torch.tensor(ts, dtype=torch.float32, device=dev)
        w = np.zeros(self.n_out)
        w[:used_out] = 1.0
        self.w_out = torch.tensor(w, dtype=torch.float32, device=dev)
        Xn = ((X - fm) / fs).astype(np.float32)
        Xn[:, 2 * self.n + 2:] = 0.0
        Tn = ((T - tm) / ts).astype(np.float32)
        return Xn, Tn

    # ------------------------------------------------------------------ training
    def fit(self, epochs=100, lr=1e-3, seed=0, stream=None, log=None):
        """Adam on minibatches of the collected examples (shuffled once on the host).
        Returns the loss history (one value per epoch, the last minibatch's)."""
        import torch
        Xn, Tn = self._standardise()
        rng = np.random.default_rng(seed)
        perm = rng.permutation(Xn.shape[0])
        nb = Xn.shape[0] // self.batch
        if nb < 1:
            raise ValueError("fewer examples than one minibatch")
        dev = self.fmean.device
        X = torch.tensor(Xn[perm[:nb * self.batch]], device=dev).view(nb, self.batch, -1)
        T = torch.tensor(Tn[perm[:nb * self.batch]], device=dev).view(nb, self.batch, -1)
        y = torch.empty((self.batch, self.n_out), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        hist = []
        for ep in range(epochs):
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))    # cosine decay
            for b in range(nb):
                mri_mlp_grad(self.net, X[b], T[b], self.w_out, y, loss, stream=stream)
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
        adaptive solve of it (cell_stats[:, 0], host or device)."""
        import torch
        ncell = y_in.shape[0]
        x = torch.empty((ncell, self.n_in), dtype=torch.float32, device=y_in.device)
        zero = torch.zeros(self.n_in, dtype=torch.float32, device=y_in.device)
        one = torch.ones(self.n_in, dtype=torch.float32, device=y_in.device)
        mri_learned_features(y_in, p, phi, Hstage, zero, one, x)
        acc = accepted.cpu().numpy() if hasattr(accepted, "cpu") else np.asarray(accepted)
        k = np.log2(n_substeps(Hstage, h) / np.maximum(acc, 1).astype(np.float64))
        self.records.append((x, k))

    def fit(self, epochs=100, lr=1e-3, seed=0, stream=None):
        import torch
        X = torch.cat([r[0] for r in self.records]).cpu().numpy().astype(np.float64)
        k = np.concatenate([r[1] for r in self.records])
        fm, fs = X.mean(0), X.std(0)
        fs[fs < 1e-12] = 1.0
        self.kmean, self.kstd = float(k.mean()), float(max(k.std(), 1e-6))
        dev = self.fmean.device
        self.fmean = torch.tensor(fm, dtype=torch.float32, device=dev)
        self.finv = torch.tensor(1.0 / fs, dtype=torch.float32, device=dev)
        Xn = ((X - fm) / fs).astype(np.float32)
        Xn[:, 2 * self.n + 2:] = 0.0
        Tn = np.zeros((Xn.shape[0], self.n_out), dtype=np.float32)
        Tn[:, 0] = (k - self.kmean) / self.kstd
        perm = np.random.default_rng(seed).permutation(Xn.shape[0])
        nb = Xn.shape[0] // self.batch
        if nb < 1:
            raise ValueError("fewer examples than one minibatch")
        Xd = torch.tensor(Xn[perm[:nb * self.batch]], device=dev).view(nb, self.batch, -1)
        Td = torch.tensor(Tn[perm[:nb * self.batch]], device=dev).view(nb, self.batch, -1)
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
