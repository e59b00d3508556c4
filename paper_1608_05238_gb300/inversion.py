"""Gradient-based reconstruction of mu_a and/or mu_s from absorbed-energy data (Sec. 6).

The paper reconstructs mu_a (Sec. 6.1) and mu_s (Sec. 6.2) by gradient descent on the error
functional eps (Eq. 2), with the functional gradients of Sec. 5 (Eqs. 22, 28) from one forward
and one adjoint MC run per iteration, a line search that accepts a step once eps has decreased
sufficiently (Eq. 30) and a stop once the relative decrease of eps falls below a tolerance
(Eq. 29).  This driver does that on top of the differentiable forward model (autograd.py):

* the gradient comes from ``eps.backward()`` through ``HFromMu`` / ``EpsFromH`` (forward MC,
  adjoint MC, FP64 gradient combine, all in the CUDA library);
* the line search is backtracking: start from the previous accepted step times ``grow``, shrink
  by ``nu`` until eps(mu - alpha g) <= eps(mu) - c1 alpha |g|^2; its trial forward runs reuse
  the iteration's seed (common random numbers), so a trial is compared with the same packets'
  estimate of eps at mu and MC noise does not decide the comparison;
* mu stays positive (mu_a >= mu_floor, mu_s >= mu_floor);
* optionally (``precondition=True``, mu_a only; not in the paper) the mu_a step is scaled per
  pixel by 1 / (dx^2 Phi_i^2), the curvature of the local part of eps, dx^2 (H^meas - mu_a Phi)^2 / 2,
  in mu_a_i: the descent direction is then (H^meas - H)_i / Phi_i plus the scaled non-local part,
  so pixels deep in the medium move as fast as those near the source.  The line search then uses
  the directional derivative g.d instead of |g|^2.

The step update itself (mu - alpha g, clamp) is a handful of torch elementwise operations: the
driver is plumbing around the MC gradient, which is where the time goes.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field, replace

import torch

from .autograd import EpsFromH, HFromMu, MCSpec


@dataclass
class Iteration:
    it: int
    eps: float
    step: float
    trials: int
    seconds: float
    rel_err_mua: float | None = None
    rel_err_mus: float | None = None


@dataclass
class InversionResult:
    mua: torch.Tensor
    mus: torch.Tensor
    history: list = field(default_factory=list)
    converged: bool = False


def mean_relative_error(est: torch.Tensor, true: torch.Tensor) -> float:
    """Mean over the domain of |mu_true - mu_est| / mu_true (the paper's reconstruction metric)."""
    return float(((est.double() - true.double()).abs() / true.double()).mean())


def _eps_and_grad(mua, mus, Hmeas, spec, want_a, want_s):
    a = mua.clone().requires_grad_(want_a)
    s = mus.clone().requires_grad_(want_s)
    H = HFromMu.apply(a, s, spec)
    eps = EpsFromH.apply(H, Hmeas, spec.dx)
    eps.backward()
    return float(eps.detach()), (a.grad if want_a else None), (s.grad if want_s else None), H.detach()


def _eps(mua, mus, Hmeas, spec):
    with torch.no_grad():
        return float(EpsFromH.apply(HFromMu.apply(mua, mus, spec), Hmeas, spec.dx))


def invert(mua0: torch.Tensor, mus0: torch.Tensor, Hmeas: torch.Tensor, spec: MCSpec, unknowns=("mua",),
           iters: int = 20, tol: float = 1e-5, step0: float | None = None, nu: float = 0.2, grow: float = 2.0,
           c1: float = 1e-4, max_trials: int = 12, mu_floor: float = 1e-6, mua_true=None, mus_true=None,
           seed0: int = 1, precondition: bool = False) -> InversionResult:
    """Reconstruct ``unknowns`` (a subset of ("mua", "mus")) from H^meas; the others stay fixed.

    ``step0`` defaults to the step that changes the unknowns by 10 % of their norm on the first
    iteration (1, a full fixed-point-like step, with ``precondition``).  Returns the estimates and one ``Iteration`` record per accepted step.
    """
    want_a, want_s = "mua" in unknowns, "mus" in unknowns
    mua, mus = mua0.detach().clone(), mus0.detach().clone()
    res = InversionResult(mua, mus)
    alpha = step0
    t0 = time.perf_counter()
    for it in range(iters):
        s_it = replace(spec, seed=seed0 + 1009 * it, adjoint_seed=seed0 + 1009 * it + 1)
        eps, ga, gs, H = _eps_and_grad(mua, mus, Hmeas, s_it, want_a, want_s)
        da = None
        if want_a:
            da = -ga
            if precondition:  # 1 / (dx^2 Phi^2), Phi = H / mu_a = a_0
                phi = H / mua
                da = da / (float(spec.dx) ** 2 * phi * phi).clamp_min(1e-30)
        ds = -gs if want_s else None
        slope = -sum(float((g.double() * d.double()).sum()) for g, d in ((ga, da), (gs, ds)) if g is not None)
        if slope <= 0.0:
            res.converged = True
            break
        if alpha is None:
            norm_mu = sum(float((m.double() ** 2).sum()) for m, w in ((mua, want_a), (mus, want_s)) if w) ** 0.5
            norm_d = sum(float((d.double() ** 2).sum()) for d in (da, ds) if d is not None) ** 0.5
            alpha = (1.0 if precondition else 0.1 * norm_mu / norm_d)
        else:
            alpha = min(alpha * grow, 1.0) if precondition else alpha * grow
        accepted = False
        for trial in range(1, max_trials + 1):
            na = (mua + alpha * da).clamp_min(mu_floor) if want_a else mua
            ns = (mus + alpha * ds).clamp_min(mu_floor) if want_s else mus
            e_new = _eps(na, ns, Hmeas, s_it)
            if e_new <= eps - c1 * alpha * slope:
                accepted = True
                break
            alpha *= nu
        if not accepted:
            res.converged = True  # no sufficient decrease at the smallest trial step
            break
        mua, mus = na, ns
        torch.cuda.synchronize()
        rec = Iteration(it, e_new, alpha, trial, time.perf_counter() - t0)
        if mua_true is not None:
            rec.rel_err_mua = mean_relative_error(mua, mua_true)
        if mus_true is not None:
            rec.rel_err_mus = mean_relative_error(mus, mus_true)
        res.history.append(rec)
        if eps - e_new <= tol * eps:  # relative decrease below tol (same packets on both sides)
            res.converged = True
            break
    res.mua, res.mus = mua, mus
    return res
