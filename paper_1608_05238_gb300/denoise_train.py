"""Training data from the method itself, training and evaluation of the harmonic-map denoiser.

Pairs are (low-count, high-count) forward harmonic maps of the same random inclusion phantom,
both produced by the batched forward MC (mc_run_batch) with independent packets; the high-count
map is the training target and, on held-out phantoms, the yardstick of the denoiser's error.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mcr, workloads
from .denoiser import UNet, sample_scale


def training_medium(n: int, dx: float, seed: int, vary: bool):
    """The medium of training pair ``seed``: a 3-inclusion phantom, or with ``vary`` 0-4 inclusions
    and, for half the pairs, pixel-scale lognormal noise of up to 20 % on mu_a (the noisy estimates
    a reconstruction passes through).  Input generator only."""
    if not vary:
        return workloads.inclusion_phantom(n, dx, 3, seed=seed, margin=min(2.0, 0.15 * n * dx))
    rng = np.random.default_rng(seed + 7_777_777)
    mua, mus = workloads.inclusion_phantom(n, dx, int(rng.integers(0, 5)), seed=seed, margin=min(2.0, 0.15 * n * dx))
    if rng.uniform() < 0.5:
        sig = rng.uniform(0.0, 0.2)
        mua = (mua * np.exp(sig * rng.standard_normal(mua.shape) - 0.5 * sig * sig)).astype(np.float32)
    return mua, mus


def make_pairs(n_pairs: int, n: int = 256, dx: float = 0.05, K: int = 16, n_low: int = 100_000,
               n_high: int = 10_000_000, seed0: int = 10_000, device="cuda", vary: bool = False):
    """(x, t): low- and high-count coefficient maps [n_pairs][2K+1][n][n] (fp32, device) of random
    circular-inclusion phantoms (3 inclusions, or varied media with ``vary``; g 0.9, collimated
    line source on the top edge)."""
    C = 2 * K + 1
    x = torch.empty(n_pairs, C, n, n, device=device)
    t = torch.empty_like(x)
    common = mcr.Run(K=K, n_packets=0)
    src = mcr.Source(**workloads.top_line_source(n, dx))
    dx32, g32 = float(np.float32(dx)), float(np.float32(0.9))
    for start in range(0, n_pairs, 32):
        probs = []
        for i in range(start, min(n_pairs, start + 32)):
            mua, mus = training_medium(n, dx, seed0 + i, vary)
            med = mcr.Medium(torch.from_numpy(mua).to(device), torch.from_numpy(mus).to(device), dx32, g32)
            probs.append(mcr.Problem(med, n_low, seed=seed0 + i, stream_id=0, source=src, out=x[i]))
            probs.append(mcr.Problem(med, n_high, seed=seed0 + i, stream_id=1, source=src, out=t[i]))
        mcr.run_batch(probs, common)
    mcr.check()
    return x, t


def make_adjoint_pairs(n_pairs: int, n: int = 256, dx: float = 0.05, K: int = 16, n_low: int = 100_000,
                       n_high: int = 10_000_000, seed0: int = 50_000, device="cuda"):
    """(x, t): low- and high-count ADJOINT coefficient maps (Sec. 4) [n_pairs][2K+1][n][n] of signed
    sources shaped like a reconstruction's q* (``workloads.residual_source``) in varied media, by
    the batched launch (adjoint problems: mc_run_batch with qstar)."""
    C = 2 * K + 1
    x = torch.empty(n_pairs, C, n, n, device=device)
    t = torch.empty_like(x)
    common = mcr.Run(K=K, n_packets=0)
    dx32, g32 = float(np.float32(dx)), float(np.float32(0.9))
    for start in range(0, n_pairs, 32):
        probs, keep = [], []
        for i in range(start, min(n_pairs, start + 32)):
            mua, mus = training_medium(n, dx, seed0 + i, True)
            med = mcr.Medium(torch.from_numpy(mua).to(device), torch.from_numpy(mus).to(device), dx32, g32)
            q = torch.from_numpy(workloads.residual_source(n, dx, seed0 + i)).to(device)
            keep.append(q)
            probs.append(mcr.Problem(med, n_low, seed=seed0 + i, stream_id=1, qstar=q, out=x[i]))
            probs.append(mcr.Problem(med, n_high, seed=seed0 + i, stream_id=3, qstar=q, out=t[i]))
        mcr.run_batch(probs, common)
    mcr.check()
    return x, t


def train(net: UNet, x: torch.Tensor, t: torch.Tensor, steps: int, batch: int = 8, lr: float = 1e-3,
          seed: int = 0, log_every: int = 0):
    """Adam on random mini-batches of the pairs, cosine-decayed learning rate; returns the losses."""
    g = torch.Generator().manual_seed(seed)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, x.shape[0], (batch,), generator=g).to(x.device)
        xb, tb = x[idx].contiguous(), t[idx].contiguous()
        lr_s = lr * 0.5 * (1 + np.cos(np.pi * s / max(1, steps)))
        loss = net.train_step(xb, sample_scale(xb), tb, lr_s)
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, loss.item()))
    return losses


def relative_error(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Per-sample ||a - b|| / ||b|| over all channels and pixels."""
    d = (a - b).flatten(1).norm(dim=1)
    return d / b.flatten(1).norm(dim=1).clamp_min(1e-30)


@torch.no_grad()
def evaluate(net: UNet, x: torch.Tensor, t: torch.Tensor, batch: int = 8):
    """Mean relative L2 error of the low-count input and of the denoised output against the
    high-count target, overall and for the fluence channel a_0."""
    err_in, err_out, e0_in, e0_out = [], [], [], []
    for s in range(0, x.shape[0], batch):
        xb, tb = x[s:s + batch].contiguous(), t[s:s + batch].contiguous()
        y = net.predict(xb, sample_scale(xb)).clone()
        err_in.append(relative_error(xb, tb))
        err_out.append(relative_error(y, tb))
        e0_in.append(relative_error(xb[:, :1], tb[:, :1]))
        e0_out.append(relative_error(y[:, :1], tb[:, :1]))
    cat = lambda v: torch.cat(v).mean().item()
    return {"err_input": cat(err_in), "err_denoised": cat(err_out), "err_a0_input": cat(e0_in),
            "err_a0_denoised": cat(e0_out)}


def plain_mc_error_curve(t: torch.Tensor, counts, n: int = 256, dx: float = 0.05, K: int = 16,
                         seed0: int = 10_000, first: int = 0):
    """Error of plain (not denoised) MC against the high-count targets ``t`` of the phantoms
    ``seed0 + first + i`` as a function of the packet count, with the MC time per map.

    Returns [(packets, mean relative L2 error, mean fluence-channel error, ms per map)], the maps
    drawn with fresh packets (stream 2) so that they share none with the inputs or targets.
    """
    C = 2 * K + 1
    common = mcr.Run(K=K, n_packets=0)
    src = mcr.Source(**workloads.top_line_source(n, dx))
    dx32, g32 = float(np.float32(dx)), float(np.float32(0.9))
    meds = []
    for i in range(t.shape[0]):
        mua, mus = workloads.inclusion_phantom(n, dx, 3, seed=seed0 + first + i, margin=min(2.0, 0.15 * n * dx))
        meds.append(mcr.Medium(torch.from_numpy(mua).to(t.device), torch.from_numpy(mus).to(t.device), dx32, g32))
    out = torch.empty(t.shape[0], C, n, n, device=t.device)
    curve = []
    for m in counts:
        probs = [mcr.Problem(md, int(m), seed=seed0 + first + i, stream_id=2, source=src, out=out[i])
                 for i, md in enumerate(meds)]
        mcr.run_batch(probs, common)  # warm-up (workspace size)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mcr.run_batch(probs, common)
        b.record()
        b.synchronize()
        curve.append((int(m), relative_error(out, t).mean().item(), relative_error(out[:, :1], t[:, :1]).mean().item(),
                      a.elapsed_time(b) / t.shape[0]))
    mcr.check()
    return curve


def packets_at_error(curve, err: float, which: int = 1) -> float:
    """Packet count at which plain MC reaches ``err`` (log-log interpolation of the curve; the
    error of plain MC falls as a power of the packet count).  ``which`` 1: all channels, 2: a_0."""
    m = np.log([c[0] for c in curve])
    e = np.log([c[which] for c in curve])
    slope, icpt = np.polyfit(m, e, 1)
    return float(np.exp((np.log(err) - icpt) / slope))
