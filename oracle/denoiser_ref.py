"""Plain PyTorch CPU reference of the harmonic-map U-Net denoiser (TEST INFRASTRUCTURE ONLY).

The same architecture as the tensor-core implementation -- 4 levels (32/64/128/256 channels),
two 3x3 convolutions + ReLU per level, 2x2 average pooling, nearest 2x up-sampling, skip
concatenation [up | skip], 1x1 output head, residual output and mean squared error -- written with
torch.nn.functional on the CPU in FP32.  With ``bf16=True`` it rounds the weights, the input
and every stored activation to bfloat16 at the same points as the GPU path, so that the
comparison isolates accumulation order; gradients come from torch autograd (straight through
the roundings).  Weights are given as {name: (w [cout][taps][cin], b [cout])}.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

NAMES = ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "ma", "mb", "d2a", "d2b", "d1a", "d1b", "d0a", "d0b", "out"]


def _q(t, on):
    return t + (t.bfloat16().float() - t).detach() if on else t


def _conv(x, w, b, relu, bf16):
    cout, taps, cin = w.shape
    k = 3 if taps == 9 else 1
    w4 = _q(w, bf16).reshape(cout, k, k, cin).permute(0, 3, 1, 2)
    y = F.conv2d(x, w4, b, padding=k // 2)
    return _q(torch.relu(y), bf16) if relu else y


def forward(params, x, bf16=True):
    """params: {name: (w, b)} leaf tensors; x: [B][C][H][W] scaled input.  Returns (y, out)."""
    q = lambda t: _q(t, bf16)
    P = params
    x0 = q(x)
    c = lambda name, t, relu=True: _conv(t, P[name][0], P[name][1], relu, bf16)
    e0a = c("e0a", x0)
    e0b = c("e0b", e0a)
    e1a = c("e1a", q(F.avg_pool2d(e0b, 2)))
    e1b = c("e1b", e1a)
    e2a = c("e2a", q(F.avg_pool2d(e1b, 2)))
    e2b = c("e2b", e2a)
    ma = c("ma", q(F.avg_pool2d(e2b, 2)))
    mb = c("mb", ma)
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    d2a = c("d2a", torch.cat([up(mb), e2b], dim=1))
    d2b = c("d2b", d2a)
    d1a = c("d1a", torch.cat([up(d2b), e1b], dim=1))
    d1b = c("d1b", d1a)
    d0a = c("d0a", torch.cat([up(d1b), e0b], dim=1))
    d0b = c("d0b", d0a)
    out = c("out", d0b, relu=False)
    return x0 + out, out


def loss_and_grads(state, x, target, bf16=True):
    """MSE of the residual output against target and its gradients for every weight and bias."""
    params = {n: (w.clone().float().requires_grad_(True), b.clone().float().requires_grad_(True))
              for n, (w, b) in state.items()}
    y, _ = forward(params, x.float(), bf16)
    loss = ((y - target.float()) ** 2).mean()
    loss.backward()
    return loss.item(), y.detach(), {n: (p[0].grad, p[1].grad) for n, p in params.items()}
