"""Gradient-based reconstruction of mu_a and/or mu_s from absorbed-energy data (Sec. 6).

The paper reconstructs mu_a (Sec. 6.1) and mu_s (Sec. 6.2) by gradient descent on the error
functional eps (Eq. 2), with the functional gradients of Sec. 5 (Eqs. 22, 28) from one forward
and one adjoint MC run per iteration, a line search that accepts a step once eps has decreased
sufficiently (Eq. 30) and a stop once the relative decrease of eps falls below a tolerance
(Eq. 29).  This driver does that on top of the differentiable forward model (autograd.py):

* the gradient comes from ``eps.backward()`` through ``HFromMu`` / ``EpsFromH`` (forward MC,
  adjoint MC, FP64 gradient combine, all in the CUDA library);
* the default line search is backtracking: start from the previous accepted step times ``grow``,
  shrink until eps(mu - alpha g) <= eps(mu) - armijo alpha |g|^2; its trial forward runs reuse
  the iteration's seed (common random numbers), so a trial is compared with the same packets'
  estimate of eps at mu and MC noise does not decide the comparison;
* or (``line_search="hager_zhang"``, the paper's choice for mu_a) the Hager-Zhang line search:
  a bracketing phase, secant steps and bisection until a trial step meets the Wolfe or the
  approximate Wolfe conditions; every trial is a full gradient evaluation (forward + adjoint MC)
  on the iteration's seeds;
* ``armijo`` is the sufficient-decrease constant of Eq. 30 (the paper's nu = 0.2 for its mu_s
  reconstruction), ``shrink`` the backtracking factor (not stated in the paper; 0.2 by default)
  and ``step_bounds`` the range the backtracking step is kept in (the paper's [1e5, 1e9] for mu_s
  in its units); the stop is Eq. 29, |eps_i - eps_(i-1)| / |eps_i| < tol;
* mu stays positive (mu_a >= mu_floor, mu_s >= mu_floor);
* optionally (``precondition=True``, mu_a only; not in the paper) the mu_a step is scaled per
  pixel by 1 / (dx^2 Phi_i^2), the curvature of the local part of eps, dx^2 (H^meas - mu_a Phi)^2 / 2,
  in mu_a_i: the descent direction is then (H^meas - H)_i / Phi_i plus the scaled non-local part,
  so pixels deep in the medium move as fast as those near the source.  The line search then uses
  the directional derivative g.d instead of |g|^2.

* or (``method="lbfgs"``; the paper chose gradient descent over L-BFGS for its robustness to MC
  noise, Sec. 6) limited-memory BFGS: the direction -H g from the two-loop recursion over the
  last ``memory`` pairs s = mu_new - mu_old, y = g_new - g_old, H_0 scaled by s.y / y.y, with the
  Hager-Zhang line search starting at the unit step.  Both gradients of a pair come from the same
  packets (the iteration's seeds: g_old at the start, g_new at the accepted trial), so y holds the
  change of the gradient and not the difference of two MC noises; pairs with s.y <= 0 are skipped,
  and a direction that is not a descent direction restarts from -g.  With ``precondition`` the
  mu_a part of H_0 is the diagonal 1 / (dx^2 Phi^2) above instead of gamma I (recomputed from
  each iteration's fluence), and the line search starts at the unit step from the first
  iteration on.

Every inner product (g.d, the line-search slopes, the recursion's s.q and y.r) is ``mc_dot``: FP64
on the GPU in a fixed order.  The step update itself (mu - alpha g, clamp) and the recursion's
vector updates are a handful of torch elementwise operations: the driver is plumbing around the MC
gradient, which is where the time goes.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field, replace

import torch

from . import mcr
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
    extra: dict | None = None  # what the caller's monitor reported after the step


@dataclass
class InversionResult:
    mua: torch.Tensor
    mus: torch.Tensor
    history: list = field(default_factory=list)
    converged: bool = False


def mean_relative_error(est: torch.Tensor, true: torch.Tensor) -> float:
    """Mean over the domain of |mu_true - mu_est| / mu_true (the paper's reconstruction metric)."""
    return float(((est.double() - true.double()).abs() / true.double()).mean())


def _dot(us, vs) -> float:
    """sum over the (non-None) tensor pairs of u.v, each by mc_dot (FP64 on the GPU, fixed order)."""
    return sum(float(mcr.dot(u.contiguous(), v.contiguous())) for u, v in zip(us, vs)
               if u is not None and v is not None)


def lbfgs_direction(g: list, pairs: list, dot=_dot, h0: list | None = None) -> list:
    """-H g by the L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4): ``g`` a list of
    tensors (None entries skipped), ``pairs`` the stored (s, y, 1 / s.y) oldest first, H_0 = gamma I
    with gamma = s.y / y.y of the newest pair (gamma = 1 without pairs), except for the entries
    where ``h0`` gives a tensor: H_0 is that diagonal there.  ``dot`` computes sums of inner
    products over the lists."""
    q = [None if t is None else t.clone() for t in g]
    alphas = []
    for s_, y_, rho in reversed(pairs):
        a = rho * dot(s_, q)
        alphas.append(a)
        q = [None if qi is None else qi - a * yi for qi, yi in zip(q, y_)]
    gamma = 1.0
    if pairs:
        s_, y_, _ = pairs[-1]
        gamma = dot(s_, y_) / dot(y_, y_)
    h0 = h0 if h0 is not None else [None] * len(q)
    r = [None if qi is None else (gamma * qi if h is None else h * qi) for qi, h in zip(q, h0)]
    for (s_, y_, rho), a in zip(pairs, reversed(alphas)):
        b = rho * dot(y_, r)
        r = [None if ri is None else ri + (a - b) * si for ri, si in zip(r, s_)]
    return [None if ri is None else -ri for ri in r]


def _eps_and_grad(mua, mus, Hmeas, spec, want_a, want_s):
    a = mua.clone().requires_grad_(want_a)
    s = mus.clone().requires_grad_(want_s)
    H = HFromMu.apply(a, s, spec)
    eps = EpsFromH.apply(H, Hmeas, spec.dx)
    eps.backward()
    return float(eps.detach()), (a.grad if want_a else None), (s.grad if want_s else None), H.detach()


def _eps(mua, mus, Hmeas, spec):
    """eps alone (the backtracking trials).  H needs only the a_0 map, and a_0's tally (each
    segment's track weight, rounded to the fixed-point quantum, which does not depend on K) and the
    packets' random numbers are the same at every K, so a K = 0 run gives the same eps bit for bit,
    at a fraction of the cost -- except through a denoiser, which maps all channels jointly."""
    if spec.denoiser is None:
        spec = replace(spec, K=0)
    with torch.no_grad():
        return float(EpsFromH.apply(HFromMu.apply(mua, mus, spec), Hmeas, spec.dx))


@dataclass
class HZParams:
    """Constants of the Hager-Zhang line search (their published defaults): Wolfe constants delta
    and sigma, the approximate-Wolfe tolerance epsilon |phi(0)|, the bisection point theta, the
    required interval shrink gamma, the bracket growth rho, and an evaluation budget."""
    delta: float = 0.1
    sigma: float = 0.9
    epsilon: float = 1e-6
    theta: float = 0.5
    gamma: float = 0.66
    rho: float = 5.0
    max_evals: int = 10


class _Accept(Exception):
    pass


class _OutOfEvals(Exception):
    pass


def _secant(a, ga, b, gb):
    return (a * gb - b * ga) / (gb - ga) if gb != ga else 0.5 * (a + b)


def hager_zhang(phi, f0: float, g0: float, c: float, p: HZParams = HZParams()):
    """Hager-Zhang line search on phi(alpha) -> (value, slope) from phi(0) = f0, phi'(0) = g0 < 0
    and the initial trial step c > 0.  Returns (alpha, phi(alpha), phi'(alpha), evaluations) for
    the first evaluated step that meets the Wolfe conditions
        phi(a) - f0 <= delta a g0   and   phi'(a) >= sigma g0
    or the approximate Wolfe conditions
        (2 delta - 1) g0 >= phi'(a) >= sigma g0   and   phi(a) <= f0 + epsilon |f0|;
    when the budget runs out first, the evaluated step with the lowest value among those with a
    sufficient decrease, else alpha = None."""
    eps_k = p.epsilon * abs(f0)
    vals = {0.0: (f0, g0)}
    n = [0]

    def ev(a):
        if a in vals:
            return vals[a]
        if n[0] >= p.max_evals:
            raise _OutOfEvals
        f, g = phi(a)
        n[0] += 1
        vals[a] = (f, g)
        wolfe = f - f0 <= p.delta * a * g0 and g >= p.sigma * g0
        approx = (2 * p.delta - 1) * g0 >= g >= p.sigma * g0 and f <= f0 + eps_k
        if wolfe or approx:
            raise _Accept(a)
        return f, g

    def bisect(a, b):  # a: slope < 0, value <= f0 + eps_k; b: slope < 0, value above it
        for _ in range(64):
            d = (1 - p.theta) * a + p.theta * b
            fd, gd = ev(d)
            if gd >= 0:
                return a, d
            if fd <= f0 + eps_k:
                a = d
            else:
                b = d
        return a, b

    def update(a, b, c):
        if not a < c < b:
            return a, b
        fc, gc = ev(c)
        if gc >= 0:
            return a, c
        if fc <= f0 + eps_k:
            return c, b
        return bisect(a, c)

    def secant2(a, b):
        c = _secant(a, vals[a][1], b, vals[b][1])
        A, B = update(a, b, c)
        if c == B:
            return update(A, B, _secant(b, vals[b][1], B, vals[B][1]))
        if c == A:
            return update(A, B, _secant(a, vals[a][1], A, vals[A][1]))
        return A, B

    def bracket(c):
        good = 0.0  # the largest trial so far with a negative slope and a value <= f0 + eps_k
        for _ in range(64):
            fc, gc = ev(c)
            if gc >= 0:
                return good, c
            if fc > f0 + eps_k:
                return bisect(0.0, c)
            good, c = c, c * p.rho
        return good, c

    try:
        a, b = bracket(c)
        for _ in range(64):
            A, B = secant2(a, b)
            if B - A > p.gamma * (b - a):
                A, B = update(A, B, 0.5 * (A + B))
            if B - A <= 1e-12 * max(B, 1e-300):
                break
            a, b = A, B
    except _Accept as e:
        alpha = e.args[0]
        return alpha, vals[alpha][0], vals[alpha][1], n[0]
    except _OutOfEvals:
        pass
    good = [(f, a) for a, (f, g) in vals.items() if a > 0 and f <= f0 + p.delta * a * g0]
    if good:
        f, a = min(good)
        return a, f, vals[a][1], n[0]
    return None, f0, g0, n[0]


def invert(mua0: torch.Tensor, mus0: torch.Tensor, Hmeas: torch.Tensor, spec: MCSpec, unknowns=("mua",),
           iters: int = 20, tol: float = 1e-5, line_search: str = "backtracking", step0: float | None = None,
           shrink: float = 0.2, grow: float = 2.0, armijo: float = 1e-4, step_bounds: tuple | None = None,
           max_trials: int = 12, hz: HZParams | None = None, mu_floor: float = 1e-6, mua_true=None, mus_true=None,
           seed0: int = 1, precondition: bool = False, method: str = "gd", memory: int = 5,
           monitor=None) -> InversionResult:
    """Reconstruct ``unknowns`` (a subset of ("mua", "mus")) from H^meas; the others stay fixed.

    ``step0`` defaults to the step that changes the unknowns by 10 % of their norm on the first
    iteration (1, a full fixed-point-like step, with ``precondition``; for the Hager-Zhang search
    its first trial is 0.01 max|mu| / max|d|, or 1 with ``precondition``).  Returns the estimates and one ``Iteration``
    record per accepted step (``trials`` = MC evaluations of the line search; ``extra`` =
    ``monitor(mua, mus)`` after the step, when a monitor is given).
    """
    if line_search not in ("backtracking", "hager_zhang"):
        raise ValueError(f"line_search must be 'backtracking' or 'hager_zhang', not {line_search!r}")
    if method not in ("gd", "lbfgs"):
        raise ValueError(f"method must be 'gd' or 'lbfgs', not {method!r}")
    if method == "lbfgs":
        line_search = "hager_zhang"  # its trials yield the gradients the pairs need
    pairs = []
    want_a, want_s = "mua" in unknowns, "mus" in unknowns
    mua, mus = mua0.detach().clone(), mus0.detach().clone()
    res = InversionResult(mua, mus)
    alpha = step0
    lo, hi = step_bounds if step_bounds is not None else (0.0, float("inf"))
    hzp = hz or HZParams()
    t0 = time.perf_counter()
    for it in range(iters):
        s_it = replace(spec, seed=seed0 + 1009 * it, adjoint_seed=seed0 + 1009 * it + 1)
        eps, ga, gs, H = _eps_and_grad(mua, mus, Hmeas, s_it, want_a, want_s)
        da, pa = None, None
        if want_a:
            da = -ga
            if precondition:  # 1 / (dx^2 Phi^2), Phi = H / mu_a = a_0
                phi = H / mua
                pa = 1.0 / (float(spec.dx) ** 2 * phi * phi).clamp_min(1e-30)
                da = da * pa
        ds = -gs if want_s else None
        if method == "lbfgs" and pairs:
            steepest = (da, ds)
            da, ds = lbfgs_direction([ga, gs], pairs, h0=[pa, None])
            if -_dot([ga, gs], [da, ds]) <= 0.0:  # not a descent direction: restart from -g (or -P g)
                pairs.clear()
                da, ds = steepest
        slope = -_dot([ga, gs], [da, ds])
        if slope <= 0.0:
            res.converged = True
            break

        def step_to(a):
            na = (mua + a * da).clamp_min(mu_floor) if want_a else mua
            ns = (mus + a * ds).clamp_min(mu_floor) if want_s else mus
            return na, ns

        if line_search == "hager_zhang":
            if method == "lbfgs" and (pairs or precondition):
                c = 1.0  # the quasi-Newton step (the preconditioned full step before any pair)
            elif alpha is None and precondition:
                c = 1.0  # the preconditioned full step
            elif alpha is None or method == "lbfgs":
                amax = max(float(m.abs().max()) for m, w in ((mua, want_a), (mus, want_s)) if w)
                dmax = max(float(d.abs().max()) for d in (da, ds) if d is not None)
                c = 0.01 * amax / dmax
            else:
                c = 2.0 * alpha
            trial_grads = {}

            def phi_fn(a):
                na, ns = step_to(a)
                e, ga2, gs2, _ = _eps_and_grad(na, ns, Hmeas, s_it, want_a, want_s)
                trial_grads[a] = (ga2, gs2)
                return e, _dot([ga2, gs2], [da, ds])

            a_acc, e_new, _, trial = hager_zhang(phi_fn, eps, -slope, c, hzp)
            if a_acc is None:
                res.converged = True  # no step with a sufficient decrease within the budget
                break
            alpha = a_acc
            na, ns = step_to(alpha)
            if method == "lbfgs":  # the pair from gradients of the same packets
                ga_n, gs_n = trial_grads[alpha]
                s_ = [(na - mua) if want_a else None, (ns - mus) if want_s else None]
                y_ = [(ga_n - ga) if want_a else None, (gs_n - gs) if want_s else None]
                sy = _dot(s_, y_)
                if sy > 1e-12 * (_dot(s_, s_) * _dot(y_, y_)) ** 0.5:
                    pairs.append((s_, y_, 1.0 / sy))
                    del pairs[:-memory]
        else:
            if alpha is None:
                norm_mu = sum(float((m.double() ** 2).sum()) for m, w in ((mua, want_a), (mus, want_s)) if w) ** 0.5
                norm_d = sum(float((d.double() ** 2).sum()) for d in (da, ds) if d is not None) ** 0.5
                alpha = (1.0 if precondition else 0.1 * norm_mu / norm_d)
            else:
                alpha = min(alpha * grow, 1.0) if precondition else alpha * grow
            alpha = min(max(alpha, lo), hi)
            accepted = False
            for trial in range(1, max_trials + 1):
                na, ns = step_to(alpha)
                e_new = _eps(na, ns, Hmeas, s_it)
                if e_new <= eps - armijo * alpha * slope:  # Eq. 30
                    accepted = True
                    break
                if alpha * shrink < lo:
                    break
                alpha *= shrink
            if not accepted:
                res.converged = True  # no sufficient decrease down to the smallest allowed step
                break
        mua, mus = na, ns
        torch.cuda.synchronize()
        rec = Iteration(it, e_new, alpha, trial, time.perf_counter() - t0)
        if mua_true is not None:
            rec.rel_err_mua = mean_relative_error(mua, mua_true)
        if mus_true is not None:
            rec.rel_err_mus = mean_relative_error(mus, mus_true)
        if monitor is not None:
            rec.extra = monitor(mua, mus)
        res.history.append(rec)
        if abs(e_new - eps) <= tol * abs(e_new):  # Eq. 29 (both values from the same packets)
            res.converged = True
            break
    res.mua, res.mus = mua, mus
    return res
