"""Learned tile-error predictor (an extension; the paper has no counterpart).

A 3-layer MLP (16 -> 128 -> 128 -> 1, ReLU; bf16 weights, fp32 accumulate)
run by the library's own kernels predicts log(1 + mean tile error) from
per-tile features, so tile selection can use fresh predictions for views
whose error maps are stale instead of a dense refresh render.  Master weights
are fp32 (packed W1 | b1 | W2 | b2 | W3 | b3); the kernels read bf16 copies.
"""
from __future__ import annotations

import math

import torch

from . import binding as B

IN, HID = 16, 128


class TileErrorMLP:
    def __init__(self, device="cuda", seed: int = 0, lr: float = 1e-3):
        g = torch.Generator().manual_seed(seed)
        n = B.mlp_param_count()
        p = torch.zeros(n)          # biases start at zero
        sl = self._slices()
        for name, fan_in in (("W1", IN), ("W2", HID), ("W3", HID)):
            k = sl[name].stop - sl[name].start
            bound = math.sqrt(6.0 / fan_in)          # He-uniform for ReLU layers
            p[sl[name]] = (torch.rand(k, generator=g) * 2 - 1) * bound
        self.params = p.to(device)
        self.m = torch.zeros(n, device=device)
        self.v = torch.zeros(n, device=device)
        self.grads = torch.zeros(n, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.step_count = 0
        self.lr = lr
        self.w1 = torch.zeros(HID * IN, dtype=torch.int16, device=device)
        self.w2 = torch.zeros(HID * HID, dtype=torch.int16, device=device)
        self.w3 = torch.zeros(HID, dtype=torch.int16, device=device)
        self._refresh_bf16()

    # views into the packed master vector
    def _slices(self):
        o1 = HID * IN
        o2 = o1 + HID
        o3 = o2 + HID * HID
        o4 = o3 + HID
        o5 = o4 + HID
        return dict(W1=slice(0, o1), b1=slice(o1, o2), W2=slice(o2, o3), b2=slice(o3, o4), W3=slice(o4, o5),
                    b3=slice(o5, o5 + 1))

    def _refresh_bf16(self):
        sl = self._slices()
        for name, dst in (("W1", self.w1), ("W2", self.w2), ("W3", self.w3)):
            dst.copy_(self.params[sl[name]].to(torch.bfloat16).view(torch.int16))

    def net(self) -> dict:
        sl = self._slices()
        return dict(w1=self.w1, w2=self.w2, w3=self.w3, b1=self.params[sl["b1"]], b2=self.params[sl["b2"]],
                    b3=self.params[sl["b3"]])

    def weights_fp(self) -> dict:
        """Master weights as float64 numpy arrays (for checks)."""
        sl = self._slices()
        p = self.params.double().cpu().numpy()
        return dict(W1=p[sl["W1"]].reshape(HID, IN), b1=p[sl["b1"]], W2=p[sl["W2"]].reshape(HID, HID),
                    b2=p[sl["b2"]], W3=p[sl["W3"]], b3=p[sl["b3"]])

    def predict(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty(x.shape[0], device=x.device)
        B.mlp_forward(self.net(), x.contiguous(), y)
        return y

    def train_step(self, x: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
        """One Adam step on mean (y - t)^2 / 2; returns the loss (device)."""
        R = x.shape[0]
        x = x.contiguous()
        y = torch.empty(R, device=x.device)
        h1 = torch.empty(R, HID, dtype=torch.int16, device=x.device)
        h2 = torch.empty(R, HID, dtype=torch.int16, device=x.device)
        B.mlp_forward(self.net(), x, y, h1, h2)
        B.mlp_backward(self.net(), x, h1, h2, y, target.contiguous(), self.grads, self.loss)
        self.step_count += 1
        B.mlp_adam(self.params, self.grads, self.m, self.v, self.step_count, self.lr, 0.9, 0.999, 1e-8, self.net())
        return self.loss
