"""Learned initial guess for consecutive frames (driver over the C ABI).

The network predicts the change of the first-step charges q^b between consecutive MD
frames from per-atom features of the potential; PCG then starts from
q_prev + scale * net(features) instead of the previous step's charges (Eq. 26).  Every
numerical step runs in libcpm.so kernels (features, forward, gradient, Adam, guess);
this module only orders the calls and keeps the device buffers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import cpm

N_FEATURES = 32
N_PARAMS = 10497


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


class LearnedGuess:
    """Parameters, Adam state and feature normalisation of one guess network."""

    def __init__(self, ctx: cpm.Context, seed: int = 0, bf16: bool = True):
        import torch
        self.ctx = ctx
        self.lib = ctx.lib
        self.bf16 = 1 if bf16 else 0
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.params = torch.empty(N_PARAMS, dtype=torch.float32, device=self.dev)
        self.ctx._check(self.lib.cpm_guess_init(self.ctx.h, ctypes.c_uint64(seed),
                                                _vp(self.params)))
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.norm = torch.cat([torch.zeros(N_FEATURES), torch.ones(N_FEATURES)]).to(self.dev)
        self.target_scale = 1.0
        self.step = 0

    # -- kernels --------------------------------------------------------------------
    def features(self, b, b_prev, chi):
        import torch
        frames, n = int(b.shape[0]), int(b.shape[1])
        feat = torch.empty((frames, n, N_FEATURES), dtype=torch.float32, device=self.dev)
        self.ctx._check(self.lib.cpm_guess_features(self.ctx.h, frames, _vp(b), _vp(b_prev),
                                                    _vp(chi), _vp(feat)))
        return feat

    def forward(self, feat):
        import torch
        s = feat.numel() // N_FEATURES
        out = torch.empty(s, dtype=torch.float32, device=self.dev)
        self.ctx._check(self.lib.cpm_mlp_forward(self.ctx.h, _vp(self.params), _vp(self.norm),
                                                 self.bf16, ctypes.c_int64(s), _vp(feat),
                                                 _vp(out)))
        return out

    def gradient(self, feat, target):
        s = feat.numel() // N_FEATURES
        self.ctx._check(self.lib.cpm_mlp_grad(self.ctx.h, _vp(self.params), _vp(self.norm),
                                              self.bf16, ctypes.c_int64(s), _vp(feat),
                                              _vp(target), _vp(self.grad), _vp(self.loss)))
        return float(self.loss.item()) / s

    def adam(self, lr):
        self.step += 1
        self.ctx._check(self.lib.cpm_mlp_adam(self.ctx.h, _vp(self.params), _vp(self.m),
                                              _vp(self.v), _vp(self.grad), self.step,
                                              ctypes.c_float(lr)))

    def train_step(self, feat, target, lr):
        """Gradient and Adam step in one library call; returns the batch's mean squared
        error before the step."""
        s = feat.numel() // N_FEATURES
        self.step += 1
        loss = ctypes.c_double(0.0)
        self.ctx._check(self.lib.cpm_guess_train_step(
            self.ctx.h, _vp(self.params), _vp(self.norm), self.bf16, ctypes.c_int64(s),
            _vp(feat), _vp(target), _vp(self.m), _vp(self.v), _vp(self.grad), _vp(self.loss),
            self.step, ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value

    def guess(self, feat, q_prev):
        import torch
        y = self.forward(feat)
        q0 = torch.empty_like(q_prev)
        self.ctx._check(self.lib.cpm_guess_apply(self.ctx.h, ctypes.c_int64(q_prev.numel()),
                                                 _vp(y), ctypes.c_float(self.target_scale),
                                                 _vp(q_prev), _vp(q0)))
        return q0

    def guess_frames(self, b, b_prev, chi, q_prev):
        """Features, network and q0 = q_prev + scale * net in one library call."""
        import torch
        frames = int(b.shape[0])
        q0 = torch.empty_like(q_prev)
        self.ctx._check(self.lib.cpm_guess(self.ctx.h, _vp(self.params), _vp(self.norm),
                                           self.bf16, frames, _vp(b), _vp(b_prev), _vp(chi),
                                           ctypes.c_float(self.target_scale), _vp(q_prev),
                                           _vp(q0)))
        return q0

    # -- training -------------------------------------------------------------------
    def set_normalisation(self, feat, target):
        """Per-feature mean / inverse deviation and the target scale from device samples
        feat [S, 32] and target [S] (float32), by cpm_guess_norm."""
        feat = feat.contiguous()
        target = target.to(feat.dtype).contiguous()
        ts = ctypes.c_float(1.0)
        self.ctx._check(self.lib.cpm_guess_norm(self.ctx.h, ctypes.c_int64(feat.shape[0]),
                                                _vp(feat), _vp(target), _vp(self.norm),
                                                ctypes.byref(ts)))
        self.target_scale = float(ts.value)

    def save(self, path: str):
        """The trained network (parameters, normalisation, target scale) to a file."""
        st = self.lib.cpm_guess_save(path.encode(), _vp(self.params), _vp(self.norm),
                                     ctypes.c_float(self.target_scale))
        if st != cpm.CPM_OK:
            raise cpm.CpmError(st, f"cpm_guess_save: cannot write {path}")

    def load(self, path: str):
        """A network written by save()."""
        ts = ctypes.c_float(1.0)
        st = self.lib.cpm_guess_load(path.encode(), _vp(self.params), _vp(self.norm),
                                     ctypes.byref(ts))
        if st != cpm.CPM_OK:
            raise cpm.CpmError(st, f"cpm_guess_load: {path} is not a valid guess file")
        self.target_scale = float(ts.value)

    def train(self, feat, target_q, epochs=3, batch=32768, lr=2e-3, seed=0, log=None):
        """Adam on the mean squared error of net(features) vs Delta q^b / target_scale.
        feat [S, 32] and target_q [S] are device tensors (float32); samples are visited in
        a seeded random order of contiguous blocks."""
        import torch
        s = feat.shape[0]
        target = (target_q / self.target_scale).to(torch.float32).contiguous()
        rng = np.random.default_rng(seed)
        starts = np.arange(0, s, batch)
        losses = []
        for ep in range(epochs):
            for b0 in rng.permutation(starts):
                b1 = min(s, b0 + batch)
                losses.append(self.train_step(feat[b0:b1], target[b0:b1], lr))
            if log:
                log(f"epoch {ep}: loss {np.mean(losses[-len(starts):]):.4e}")
        return losses
