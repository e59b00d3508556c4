"""The learned part inside the method: denoised low-count forward and adjoint harmonic maps feed the
functional gradient, with full-count MC as the judge of the denoiser's error and its fallback.

A gradient evaluation of Secs. 4-5 needs the forward coefficients (a_n, b_n) and the adjoint
coefficients (a*_n, b*_n) of every pixel (Eqs. 22, 28).  Their MC noise falls like 1/sqrt(N_p), so
the packet count sets the cost.  Here both runs use a low count and each map goes through a U-Net
trained on pairs the MC itself generates (one network for forward maps, one for adjoint maps:
their sources and statistics differ), and the denoised maps take the MC maps' place in H = mu_a a_0
and in the gradient combine.  (The paper has no learned part.)

Judge and fallback: every ``judge_every``-th evaluation (and, with ``judge_first``, the first) of
each kind also runs an independent MC of ``n_judge`` packets (default ``n_full``; a count ~10x the
low one already measures the low-count map's error to ~5 %) for the same medium and source,
measures the relative L2 error of the denoised map and of the raw low-count map against it, and
uses that map for the evaluation.  If the denoised map is worse than ``max_rel_err`` -- or worse
than the raw low-count map it started from -- the denoiser is switched off for good
(``fallback``) and every later evaluation runs full-count MC (``n_full`` packets).  The judgments
are kept in ``history``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from .denoiser import UNet, sample_scale


def _rel(a: torch.Tensor, b: torch.Tensor) -> float:
    """||a - b|| / ||b|| over all channels and pixels (a diagnostic of the judge)."""
    return float((a - b).norm() / b.norm().clamp_min(1e-30))


@dataclass
class Denoiser:
    """Forward and adjoint U-Nets (in_ch = 2K+1 of the maps they denoise) and the judge's settings."""
    fwd: UNet
    adj: UNet
    n_full: int = 10_000_000       # packets of a fallback run
    n_judge: int | None = None     # packets of a judging run (default n_full)
    judge_every: int = 0           # 0: judge only the first evaluation of each kind (if judge_first)
    judge_first: bool = True
    max_rel_err: float = 0.25      # switch to full-count MC when the denoised map is worse than this
    fallback: bool = False
    history: list = field(default_factory=list)
    _calls: dict = field(default_factory=lambda: {"forward": 0, "adjoint": 0})

    def _net(self, kind: str) -> UNet:
        return self.fwd if kind == "forward" else self.adj

    def denoise(self, kind: str, coeff: torch.Tensor) -> torch.Tensor:
        """Denoised [2K+1, nz, nx] map from a low-count one (a batch of one through the U-Net)."""
        x = coeff.unsqueeze(0).contiguous()
        return self._net(kind).predict(x, sample_scale(x))[0].clone()

    def wants_judge(self, kind: str) -> bool:
        """True when this evaluation of ``kind`` is one the full-count MC judges."""
        k = self._calls[kind]
        self._calls[kind] = k + 1
        return (k == 0 and self.judge_first) or (k > 0 and self.judge_every > 0 and k % self.judge_every == 0)

    def judge(self, kind: str, low: torch.Tensor, denoised: torch.Tensor, full: torch.Tensor) -> torch.Tensor:
        """Record the errors of the denoised and the raw low-count map against the full-count map,
        switch to full-count MC if the denoiser fails, and return the map to use (the full one)."""
        e_dn, e_low = _rel(denoised, full), _rel(low, full)
        bad = not (e_dn <= self.max_rel_err and e_dn <= e_low)  # a NaN fails too
        self.history.append({"kind": kind, "call": self._calls[kind] - 1, "err_denoised": e_dn, "err_low": e_low,
                             "fallback": bad})
        if bad:
            self.fallback = True
        return full
