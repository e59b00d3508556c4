"""The reconstruction driver (Sec. 6) on the GPU: mu_a-only gradient descent with backtracking on a
small inclusion phantom, started from a uniform guess twice the background, lowers eps at every
accepted step and the mean relative error of mu_a over the domain."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from paper_1608_05238_gb300 import _build, mcr, workloads
from paper_1608_05238_gb300.autograd import MCSpec, forward_coefficients
from paper_1608_05238_gb300.inversion import invert, mean_relative_error
from parity_util import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()


def test_mua_reconstruction_reduces_eps_and_error():
    n, dx = 64, 0.1
    mua_t, mus_t = workloads.inclusion_phantom(n, dx, 2, seed=7, margin=1.5, radius=(0.6, 1.2),
                                               mus_range=(10.0, 10.0))
    src = mcr.Source(**workloads.top_line_source(n, dx))
    g = f32(0.9)
    dev = torch.device("cuda")
    mua_true, mus = torch.from_numpy(mua_t).to(dev), torch.from_numpy(mus_t).to(dev)
    hspec = MCSpec(dx=f32(dx), g=g, sources=[src], K=0, n_packets=4_000_000, seed=99)
    Hmeas = mcr.h_eps(mcr.Medium(mua_true, mus, f32(dx), g), forward_coefficients(
        mcr.Medium(mua_true, mus, f32(dx), g), hspec))
    spec = MCSpec(dx=f32(dx), g=g, sources=[src], K=8, n_packets=2_000_000)
    mua0 = torch.full_like(mua_true, 0.02)  # background 0.01: 100 % error there
    res = invert(mua0, mus, Hmeas, spec, unknowns=("mua",), iters=10, mua_true=mua_true)
    assert len(res.history) >= 3
    e0 = mean_relative_error(mua0, mua_true)
    eps = [h.eps for h in res.history]
    errs = [h.rel_err_mua for h in res.history]
    assert all(b < a for a, b in zip(eps, eps[1:])), eps
    assert errs[-1] < 0.6 * e0, (e0, errs)
    assert torch.all(res.mua > 0) and torch.equal(res.mus, mus)


def test_preconditioned_mua_reconstruction_converges_fast():
    """With the step scaled by 1 / (dx^2 Phi^2) the reconstruction behaves like the fixed point
    mu_a <- H^meas / Phi: a few iterations bring the error down to the MC noise level."""
    n, dx = 64, 0.1
    mua_t, mus_t = workloads.inclusion_phantom(n, dx, 2, seed=7, margin=1.5, radius=(0.6, 1.2),
                                               mus_range=(10.0, 10.0))
    src = mcr.Source(**workloads.top_line_source(n, dx))
    g = f32(0.9)
    dev = torch.device("cuda")
    mua_true, mus = torch.from_numpy(mua_t).to(dev), torch.from_numpy(mus_t).to(dev)
    med = mcr.Medium(mua_true, mus, f32(dx), g)
    Hmeas = mcr.h_eps(med, forward_coefficients(med, MCSpec(dx=f32(dx), g=g, sources=[src], K=0,
                                                           n_packets=8_000_000, seed=99)))
    spec = MCSpec(dx=f32(dx), g=g, sources=[src], K=8, n_packets=2_000_000)
    mua0 = torch.full_like(mua_true, 0.02)
    res = invert(mua0, mus, Hmeas, spec, unknowns=("mua",), iters=6, mua_true=mua_true, precondition=True)
    e0 = mean_relative_error(mua0, mua_true)
    errs = [h.rel_err_mua for h in res.history]
    assert errs[-1] < 0.15 * e0, (e0, errs)


def _rect_setup(n_meas, K, n_packets):
    mua_t, mus_t, g, srcs = workloads.rect_phantom()
    dx, g = f32(0.05), f32(g)
    dev = torch.device("cuda")
    mua_t, mus_t = torch.from_numpy(mua_t).to(dev), torch.from_numpy(mus_t).to(dev)
    sources = [mcr.Source(**s) for s in srcs]
    med = mcr.Medium(mua_t, mus_t, dx, g)
    Hmeas = mcr.h_eps(med, forward_coefficients(med, MCSpec(dx=dx, g=g, sources=sources, K=0, n_packets=n_meas,
                                                            seed=1001)))
    return mua_t, mus_t, Hmeas, MCSpec(dx=dx, g=g, sources=sources, K=K, n_packets=n_packets)


def test_hager_zhang_mua_reconstruction_of_the_rectangular_inclusion():
    """Sec. 6.1's setting (rectangular inclusions, two adjacent line sources, mu_s known, start at
    the background): gradient descent with the Hager-Zhang line search brings the mean relative
    mu_a error below half its start within eight iterations and eps down by two orders."""
    mua_t, mus_t, Hmeas, spec = _rect_setup(20_000_000, 8, 2_000_000)
    mua0 = torch.full_like(mua_t, 0.01)
    res = invert(mua0, mus_t, Hmeas, spec, unknowns=("mua",), iters=8, tol=1e-9, line_search="hager_zhang",
                 mua_true=mua_t)
    e0 = mean_relative_error(mua0, mua_t)
    errs = [h.rel_err_mua for h in res.history]
    assert len(res.history) == 8, res.history
    assert res.history[-1].eps < 1e-2 * res.history[0].eps, [h.eps for h in res.history]
    assert errs[-1] < 0.5 * e0, (e0, errs)
    assert all(h.trials >= 1 for h in res.history) and torch.equal(res.mus, mus_t)


def test_backtracking_mus_reconstruction_lowers_eps_within_step_bounds():
    """Sec. 6.2's mu_s-only setting: backtracking with the Eq. 30 constant 0.2 and steps kept in
    [1e5, 1e9] lowers eps at every accepted step and moves mu_s inside the inclusion up from the
    background towards its true value."""
    mua_t, mus_t, Hmeas, spec = _rect_setup(20_000_000, 8, 2_000_000)
    mus0 = torch.full_like(mus_t, 5.0)
    res = invert(mua_t, mus0, Hmeas, spec, unknowns=("mus",), iters=8, tol=1e-5, line_search="backtracking",
                 armijo=0.2, shrink=0.5, step_bounds=(1e5, 1e9), mus_true=mus_t)
    assert len(res.history) >= 4
    assert all(1e5 <= h.step <= 1e9 for h in res.history)
    assert res.history[-1].eps < 0.5 * res.history[0].eps, [h.eps for h in res.history]
    incl = mus_t > 10
    assert float(res.mus[incl].mean()) > 5.5 and torch.equal(res.mua, mua_t)


def test_mc_dot_is_fp64_and_deterministic():
    """The inner products of the line searches: FP64 products and sums (no FP32 accumulation
    error), the same bits on every call."""
    g = torch.Generator().manual_seed(5)
    a = (torch.randn(1_000_003, generator=g) * 1e3).cuda()
    b = (torch.randn(1_000_003, generator=g) * 1e-3).cuda()
    ref = float((a.double().cpu() * b.double().cpu()).sum())
    got = [float(mcr.dot(a, b)) for _ in range(3)]
    assert got[0] == got[1] == got[2]
    assert abs(got[0] - ref) <= 1e-12 * float((a.double().abs() * b.double().abs()).sum())
    with pytest.raises(ValueError):
        mcr.dot(a, b[:10])


def test_lbfgs_mua_reconstruction_of_the_rectangular_inclusion():
    """L-BFGS (pairs from gradients of the same packets, Hager-Zhang from the unit step) on the
    Sec. 6.1 setting: eps falls by two orders and the mean relative mu_a error below half its start
    within eight iterations, mu_s untouched."""
    mua_t, mus_t, Hmeas, spec = _rect_setup(20_000_000, 8, 2_000_000)
    mua0 = torch.full_like(mua_t, 0.01)
    res = invert(mua0, mus_t, Hmeas, spec, unknowns=("mua",), iters=8, tol=1e-12, method="lbfgs", mua_true=mua_t)
    e0 = mean_relative_error(mua0, mua_t)
    errs = [h.rel_err_mua for h in res.history]
    assert len(res.history) >= 6, res.history
    assert res.history[-1].eps < 1e-2 * res.history[0].eps, [h.eps for h in res.history]
    assert errs[-1] < 0.5 * e0, (e0, errs)
    assert torch.equal(res.mus, mus_t) and torch.all(res.mua > 0)


def test_preconditioned_lbfgs_mua_reconstruction():
    """L-BFGS with the fluence preconditioner as its initial inverse Hessian (the unit step from the
    first iteration) on the 64^2 two-inclusion phantom: like the preconditioned descent it brings
    the error well below its start within a few iterations; mu_s is untouched."""
    n, dx = 64, 0.1
    mua_t, mus_t = workloads.inclusion_phantom(n, dx, 2, seed=7, margin=1.5, radius=(0.6, 1.2),
                                               mus_range=(10.0, 10.0))
    src = mcr.Source(**workloads.top_line_source(n, dx))
    g = f32(0.9)
    dev = torch.device("cuda")
    mua_true, mus = torch.from_numpy(mua_t).to(dev), torch.from_numpy(mus_t).to(dev)
    med = mcr.Medium(mua_true, mus, f32(dx), g)
    Hmeas = mcr.h_eps(med, forward_coefficients(med, MCSpec(dx=f32(dx), g=g, sources=[src], K=0,
                                                           n_packets=8_000_000, seed=99)))
    spec = MCSpec(dx=f32(dx), g=g, sources=[src], K=8, n_packets=2_000_000)
    mua0 = torch.full_like(mua_true, 0.02)
    res = invert(mua0, mus, Hmeas, spec, unknowns=("mua",), iters=6, tol=1e-12, mua_true=mua_true,
                 precondition=True, method="lbfgs")
    e0 = mean_relative_error(mua0, mua_true)
    errs = [h.rel_err_mua for h in res.history]
    assert len(res.history) >= 2, res.history
    assert errs[-1] < 0.15 * e0, (e0, errs)
    assert torch.equal(res.mus, mus) and torch.all(res.mua > 0)


def test_eps_trials_at_k0_equal_the_full_order_eps():
    """The backtracking trials evaluate eps with K = 0 runs: a_0 (and so H and eps) is the same bit
    for bit as in the run at the spec's K on the same packets."""
    from paper_1608_05238_gb300.autograd import EpsFromH, HFromMu
    from paper_1608_05238_gb300.inversion import _eps
    mua_t, mus_t, Hmeas, spec = _rect_setup(2_000_000, 12, 500_000)
    mua = torch.full_like(mua_t, 0.012)
    with torch.no_grad():
        eps_full = float(EpsFromH.apply(HFromMu.apply(mua, mus_t, spec), Hmeas, spec.dx))
    assert _eps(mua, mus_t, Hmeas, spec) == eps_full
    med = mcr.Medium(mua, mus_t, spec.dx, spec.g)
    assert torch.equal(forward_coefficients(med, replace(spec, K=0))[0], forward_coefficients(med, spec)[0])
