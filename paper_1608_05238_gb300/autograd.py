"""Differentiable forward model: ``torch.autograd.Function`` wrappers over the CUDA library.

``HFromMu.apply(mua, mus, spec)`` maps the absorption and scattering maps to the absorbed energy
H = mu_a Phi (Sec. 2) with the forward harmonic radiance MC (Sec. 3).  Its backward is the
adjoint method of Secs. 4-5: given v = dL/dH it launches the adjoint MC from
q* = -mu_a v / dx^2 (Sec. 6's q* = mu_a (H^meas - H) when L is Eq. 2's eps) and combines forward
and adjoint coefficients pixel by pixel into
    dL/dmu_a = v a_0 + dx^2 [a_0 a_0*/(2 pi) + (1/pi) sum (a_n a_n* + b_n b_n*)]      (Eq. 22)
    dL/dmu_s = dx^2 (1/pi) sum (a_n a_n* + b_n b_n*)(1 - g^n)                        (Eq. 28)
with FP64 sums.  The forward coefficients are kept for the backward pass, or -- at large K or
when they would exceed a memory budget -- recomputed from the same seeds, which reproduces them
bit for bit (fixed-point tallies do not depend on scheduling).  The adjoint source is always
built in the backward pass from the incoming gradient.

``EpsFromH.apply(H, Hmeas, dx)`` is the error functional of Eq. 2 with dL/dH = -dx^2 (H^meas - H).
Every arithmetic step runs in libmcr's kernels; autograd adds only its own bookkeeping (the seed
gradient of the scalar loss and its product with dL/dH).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import torch

from . import mcr, mcr3, shard


@dataclass
class MCSpec:
    """What the forward model runs: geometry, illumination, harmonic order and packet budgets."""
    dx: float
    g: float
    sources: list                     # mcr.Source list; their fluences add (one illumination)
    K: int
    n_packets: int                    # packets per forward source
    n_adjoint: int | None = None      # adjoint packets (default: n_packets)
    seed: int = 0
    adjoint_seed: int | None = None   # default: seed
    recompute: bool | None = None     # None: recompute when K > 32 or coeff > coeff_budget bytes
    coeff_budget: int = 256 << 20
    w_threshold: float = 1e-4
    roulette_p: float = 0.1
    max_events: int = 10_000_000
    sharded: bool = False             # split every run's packets over the ranks of torch.distributed's
                                      # default group (exact int64 all-reduce of the fixed-point sums)
    denoiser: object | None = None    # denoised.Denoiser: low-count maps through the U-Nets, judged by
                                      # (and falling back to) full-count MC

    def forward_run(self, s: int) -> mcr.Run:
        return mcr.Run(K=self.K, n_packets=self.n_packets, seed=self.seed, stream_id=2 * s,
                       w_threshold=self.w_threshold, roulette_p=self.roulette_p, max_events=self.max_events)

    def adjoint_run(self) -> mcr.Run:
        return mcr.Run(K=self.K, n_packets=self.n_adjoint or self.n_packets,
                       seed=self.seed if self.adjoint_seed is None else self.adjoint_seed, stream_id=1,
                       w_threshold=self.w_threshold, roulette_p=self.roulette_p, max_events=self.max_events)

    def should_recompute(self, nz: int, nx: int) -> bool:
        if self.denoiser is not None:  # keep the (denoised or judged) maps the forward pass used
            return False
        if self.recompute is not None:
            return bool(self.recompute)
        return self.K > 32 or (2 * self.K + 1) * nz * nx * 4 > self.coeff_budget


# seed offset of the full-count runs that judge the denoiser (packets independent of the low-count run)
JUDGE_SEED = 1_000_003


def _mc_forward(med: mcr.Medium, spec: MCSpec, n: int | None = None, seed: int | None = None) -> torch.Tensor:
    fwd = shard.forward if spec.sharded else mcr.forward
    run = lambda s: replace(spec.forward_run(s), n_packets=n or spec.n_packets,
                            seed=spec.seed if seed is None else seed)
    coeff = fwd(med, spec.sources[0], run(0))
    for s in range(1, len(spec.sources)):
        fwd(med, spec.sources[s], replace(run(s), accumulate=True), out=coeff)
    return coeff


def _mc_adjoint(med: mcr.Medium, q: torch.Tensor, spec: MCSpec, n: int | None = None,
                seed: int | None = None) -> torch.Tensor:
    run = spec.adjoint_run()
    run = replace(run, n_packets=n or run.n_packets, seed=run.seed if seed is None else seed)
    return (shard.adjoint if spec.sharded else mcr.adjoint)(med, q, run)


def _denoised(kind: str, spec: MCSpec, mc) -> torch.Tensor:
    """A map through the spec's denoiser: mc(n, seed) runs the MC; full-count MC judges and replaces
    the denoised map on judged evaluations, and after a failed judgment on every evaluation."""
    dn = spec.denoiser
    if dn.fallback:
        return mc(dn.n_full, None)
    low = mc(None, None)
    out = dn.denoise(kind, low)
    if dn.wants_judge(kind):
        out = dn.judge(kind, low, out, mc(dn.n_judge or dn.n_full, spec.seed + JUDGE_SEED))
    return out


def forward_coefficients(med: mcr.Medium, spec: MCSpec) -> torch.Tensor:
    """Forward coefficients of the whole illumination (sum over ``spec.sources``, added by the
    library's finalize kernel: the RTE is linear in the source); denoised with ``spec.denoiser``."""
    if spec.denoiser is None:
        return _mc_forward(med, spec)
    return _denoised("forward", spec, lambda n, seed: _mc_forward(med, spec, n, seed))


def adjoint_coefficients(med: mcr.Medium, q: torch.Tensor, spec: MCSpec) -> torch.Tensor:
    """Adjoint coefficients from q* (packets split over the ranks when ``spec.sharded``; denoised
    with ``spec.denoiser``)."""
    if spec.denoiser is None:
        return _mc_adjoint(med, q, spec)
    return _denoised("adjoint", spec, lambda n, seed: _mc_adjoint(med, q, spec, n, seed))


class HFromMu(torch.autograd.Function):
    """(mu_a, mu_s) -> H = mu_a Phi by forward MC; backward by adjoint MC (Secs. 3-6)."""

    @staticmethod
    def forward(ctx, mua: torch.Tensor, mus: torch.Tensor, spec: MCSpec):
        mua_c = mua.detach().contiguous()
        mus_c = mus.detach().contiguous()
        med = mcr.Medium(mua_c, mus_c, spec.dx, spec.g)
        coeff = forward_coefficients(med, spec)
        H = mcr.h_eps(med, coeff)
        recompute = spec.should_recompute(*mua_c.shape)
        ctx.spec = spec
        ctx.recompute = recompute
        if recompute:
            ctx.save_for_backward(mua_c, mus_c)
        else:
            ctx.save_for_backward(mua_c, mus_c, coeff)
        return H

    @staticmethod
    def backward(ctx, grad_H: torch.Tensor):
        spec: MCSpec = ctx.spec
        saved = ctx.saved_tensors
        mua_c, mus_c = saved[0], saved[1]
        med = mcr.Medium(mua_c, mus_c, spec.dx, spec.g)
        v = grad_H.detach().float().contiguous()
        q = mcr.adjoint_source(med, v)
        coeff_adj = adjoint_coefficients(med, q, spec)
        coeff = forward_coefficients(med, spec) if ctx.recompute else saved[2]
        d_mua, d_mus = mcr.gradient(med, coeff, coeff_adj, v, dtype=torch.float32)
        return (d_mua if ctx.needs_input_grad[0] else None, d_mus if ctx.needs_input_grad[1] else None, None)


class EpsFromH(torch.autograd.Function):
    """eps = 1/2 dx^2 sum (H^meas - H)^2 (Eq. 2, FP64) with dL/dH = -dx^2 (H^meas - H)."""

    @staticmethod
    def forward(ctx, H: torch.Tensor, Hmeas: torch.Tensor, dx: float):
        e, v = mcr.eps(H.detach().contiguous(), Hmeas.detach().contiguous(), dx)
        ctx.save_for_backward(v)
        return e

    @staticmethod
    def backward(ctx, grad_eps: torch.Tensor):
        (v,) = ctx.saved_tensors
        return v * grad_eps.to(v.dtype), None, None


def absorbed_energy(mua: torch.Tensor, mus: torch.Tensor, spec: MCSpec) -> torch.Tensor:
    """H(mu_a, mu_s), differentiable with respect to both maps."""
    return HFromMu.apply(mua, mus, spec)


def error_functional(H: torch.Tensor, Hmeas: torch.Tensor, dx: float) -> torch.Tensor:
    """Eq. 2's eps(H), differentiable with respect to H."""
    return EpsFromH.apply(H, Hmeas, dx)


# ------------------------------------------------------------------------------------------ 3D
@dataclass
class MCSpec3:
    """The 3D forward model (Sec. 3.1's spherical-harmonic form): voxel side, HG g, one source,
    order L and packet budgets."""
    dx: float
    g: float
    source: "mcr3.Source3"
    L: int
    n_packets: int
    n_adjoint: int | None = None
    seed: int = 0
    adjoint_seed: int | None = None
    recompute: bool = False           # recompute the forward coefficients in backward (same seeds)
    w_threshold: float = 1e-4
    roulette_p: float = 0.1
    max_events: int = 10_000_000

    def forward_run(self) -> mcr.Run:
        return mcr.Run(K=self.L, n_packets=self.n_packets, seed=self.seed, stream_id=0,
                       w_threshold=self.w_threshold, roulette_p=self.roulette_p, max_events=self.max_events)

    def adjoint_run(self) -> mcr.Run:
        return mcr.Run(K=self.L, n_packets=self.n_adjoint or self.n_packets,
                       seed=self.seed if self.adjoint_seed is None else self.adjoint_seed, stream_id=1,
                       w_threshold=self.w_threshold, roulette_p=self.roulette_p, max_events=self.max_events)


class HFromMu3(torch.autograd.Function):
    """(mu_a, mu_s) [nz, ny, nx] -> H = mu_a sqrt(4 pi) c_00 by 3D forward MC; backward by the 3D
    adjoint MC from q* = -mu_a v / dx^3 and the voxel combine
    dL/dmu_a = v sqrt(4 pi) c_00 + dx^3 sum c c*, dL/dmu_s = dx^3 sum (1 - g^l) c c*."""

    @staticmethod
    def forward(ctx, mua: torch.Tensor, mus: torch.Tensor, spec: MCSpec3):
        mua_c = mua.detach().contiguous()
        mus_c = mus.detach().contiguous()
        med = mcr3.Medium3(mua_c, mus_c, spec.dx, spec.g)
        coeff = mcr3.forward(med, spec.source, spec.forward_run())
        H = mcr3.h_eps(med, coeff)
        ctx.spec = spec
        if spec.recompute:
            ctx.save_for_backward(mua_c, mus_c)
        else:
            ctx.save_for_backward(mua_c, mus_c, coeff)
        return H

    @staticmethod
    def backward(ctx, grad_H: torch.Tensor):
        spec: MCSpec3 = ctx.spec
        saved = ctx.saved_tensors
        med = mcr3.Medium3(saved[0], saved[1], spec.dx, spec.g)
        v = grad_H.detach().float().contiguous()
        q = mcr3.adjoint_source(med, v)
        coeff_adj = mcr3.adjoint(med, q, spec.adjoint_run())
        coeff = mcr3.forward(med, spec.source, spec.forward_run()) if spec.recompute else saved[2]
        d_mua, d_mus = mcr3.gradient(med, coeff, coeff_adj, v, dtype=torch.float32)
        return (d_mua if ctx.needs_input_grad[0] else None, d_mus if ctx.needs_input_grad[1] else None, None)


class EpsFromH3(torch.autograd.Function):
    """eps = 1/2 dx^3 sum (H^meas - H)^2 (FP64) with dL/dH = -dx^3 (H^meas - H)."""

    @staticmethod
    def forward(ctx, H: torch.Tensor, Hmeas: torch.Tensor, dx: float):
        e, v = mcr3.eps(H.detach().contiguous(), Hmeas.detach().contiguous(), dx)
        ctx.save_for_backward(v)
        return e

    @staticmethod
    def backward(ctx, grad_eps: torch.Tensor):
        (v,) = ctx.saved_tensors
        return v * grad_eps.to(v.dtype), None, None
