"""The reconstruction driver (Sec. 6) on the GPU: mu_a-only gradient descent with backtracking on a
small inclusion phantom, started from a uniform guess twice the background, lowers eps at every
accepted step and the mean relative error of mu_a over the domain."""
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
