"""The differentiable forward model (HFromMu / EpsFromH) against the oracle and finite differences."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import RunParams
from oracle import functionals as F
from paper_1608_05238_gb300 import _build, mcr, workloads
from paper_1608_05238_gb300.autograd import EpsFromH, HFromMu, MCSpec
from parity_util import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()


def _spec(nx, dx, g, K, n, **kw):
    src = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(nx * dx), z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    return MCSpec(dx=f32(dx), g=f32(g), sources=[src], K=K, n_packets=n, **kw)


def _grads(mua, mus, Hm, spec):
    a = torch.from_numpy(mua).cuda().requires_grad_(True)
    s = torch.from_numpy(mus).cuda().requires_grad_(True)
    H = HFromMu.apply(a, s, spec)
    e = EpsFromH.apply(H, torch.from_numpy(Hm).cuda(), spec.dx)
    e.backward()
    return a.grad.double().cpu().numpy(), s.grad.double().cpu().numpy(), H.detach().cpu().numpy(), e.item()


def test_autograd_gradient_matches_oracle():
    """Autograd gradients vs the oracle's forward + adjoint runs on the same packets (Eqs. 22, 28).

    The incoming gradient v = dL/dH is a seeded input of both sides (L = sum v H), so both build
    the identical FP32 adjoint source q* = -mu_a v / dx^2 and draw the identical adjoint packets;
    the gradient then differs only by the transport's FP32 rounding and is held to the tally bar
    (1e-4 of the absolute scale in L1; 2e-4 per well-resolved pixel, a product of two tallies)."""
    nz, nx, dx, g, K, n = 40, 48, 0.1, 0.8, 8, 200_000
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=21)
    Hm = (1.4 * mua * np.exp(-np.linspace(0, 2, nz))[:, None]).astype(np.float32)
    spec = _spec(nx, dx, g, K, n, seed=3, adjoint_seed=4)
    dxo, go = f32(dx), f32(g)
    A = dxo * dxo
    rng = np.random.default_rng(41)
    v = (-A * (Hm - 0.9 * mua * np.exp(-np.linspace(0, 1.5, nz))[:, None]) *
         (1.0 + 0.3 * rng.normal(size=(nz, nx)))).astype(np.float32)

    a = torch.from_numpy(mua).cuda().requires_grad_(True)
    s_ = torch.from_numpy(mus).cuda().requires_grad_(True)
    H = HFromMu.apply(a, s_, spec)
    H.backward(torch.from_numpy(v).cuda())
    ga, gs = a.grad.double().cpu().numpy(), s_.grad.double().cpu().numpy()
    e = EpsFromH.apply(H.detach(), torch.from_numpy(Hm).cuda(), spec.dx).item()

    m64, s64 = mua.astype(np.float64), mus.astype(np.float64)
    src = spec.sources[0].as_dict()
    fo = oracle.forward(m64, s64, dxo, go, src, RunParams(K=K, n_packets=n, seed=3, stream_id=0)).coeff
    Ho = F.absorbed_energy(m64, fo)
    assert abs(e - F.error_functional(Hm, Ho, dxo)) <= 1e-3 * e
    v64 = v.astype(np.float64)
    q = F.adjoint_source(m64, v64, dxo).astype(np.float32)
    ao = oracle.adjoint(m64, s64, dxo, go, q, RunParams(K=K, n_packets=n, seed=4, stream_id=1)).coeff
    aabs = oracle.adjoint(m64, s64, dxo, go, np.abs(q), RunParams(K=K, n_packets=n, seed=4, stream_id=1)).coeff
    oa, os_ = F.dL_dmu(fo, ao, v64, dxo, go)
    # scale of each pixel's products with absolute values (the sums cancel, their terms do not)
    S = np.abs(v64 * fo[0]) + A * (np.abs(fo[0] * aabs[0]) / (2 * math.pi) +
                                   np.sum(np.abs(fo[1:]) * np.abs(aabs[1:]), axis=0) / math.pi)
    for G, O in ((ga, oa), (gs, os_)):
        assert np.sum(np.abs(G - O)) <= 1e-4 * np.sum(S)
        hi = S >= 1e-2 * S.max()
        assert np.max(np.abs(G - O)[hi] / S[hi]) <= 2e-4


def test_recompute_reproduces_stored_coefficients_bit_for_bit():
    nz, nx, dx, g = 24, 20, 0.1, 0.9
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=22)
    Hm = (0.8 * mua).astype(np.float32)
    out = []
    for rec in (False, True):
        spec = _spec(nx, dx, g, 64, 50_000, seed=9, recompute=rec)
        out.append(_grads(mua, mus, Hm, spec))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert _spec(nx, dx, g, 64, 10).should_recompute(nz, nx) and not _spec(nx, dx, g, 32, 10).should_recompute(nz, nx)


def test_mua_gradient_matches_crn_finite_differences_on_gpu():
    """CRN central differences of eps in each pixel's mu_a (trajectories do not depend on mu_a)."""
    n, dx, g = 6, 0.1, 0.5
    c = (np.arange(n) + 0.5) * dx
    X, Z = np.meshgrid(c, c)
    mua = (0.15 + 0.1 * np.sin(3 * X) * np.cos(2 * Z)).astype(np.float32)
    mus = (3.0 + 1.0 * np.cos(4 * X + Z)).astype(np.float32)
    Hm = (mua * (1.5 + np.sin(5 * X)) * np.exp(-Z)).astype(np.float32)
    spec = _spec(n, dx, g, 12, 400_000, seed=1, adjoint_seed=2, n_adjoint=2_000_000)
    ga, _, _, _ = _grads(mua, mus, Hm, spec)
    fspec = _spec(n, dx, g, 0, 400_000, seed=1)
    med_mus = torch.from_numpy(mus).cuda()
    Hm_d = torch.from_numpy(Hm).cuda()

    def eps(m):
        with torch.no_grad():
            H = HFromMu.apply(torch.from_numpy(m).cuda(), med_mus, fspec)
            return EpsFromH.apply(H, Hm_d, fspec.dx).item()

    fd = np.zeros_like(ga)
    h = 1e-3
    for idx in np.ndindex(mua.shape):
        e = np.zeros_like(mua)
        e[idx] = h
        fd[idx] = (eps(mua + e) - eps(mua - e)) / (2 * h)
    assert np.max(np.abs(ga - fd)) < 5e-3 * np.max(np.abs(fd))


def test_two_source_illumination_accumulates_in_the_library():
    """Several sources of one illumination: the library adds each run's coefficients into the
    same output (accumulate), equal to the FP32 sum of separate runs, and the autograd forward
    uses it."""
    from paper_1608_05238_gb300.autograd import forward_coefficients
    nz, nx, dx = 24, 20, 0.1
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=8)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(0.8))
    top = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(nx * dx), z1=0.0, dir_x=0.0, dir_z=1.0)
    left = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=0.0, z1=f32(nz * dx), dir_x=1.0, dir_z=0.0, power=0.5)
    spec = MCSpec(dx=f32(dx), g=f32(0.8), sources=[top, left], K=4, n_packets=50_000, seed=3)
    a = mcr.forward(med, top, spec.forward_run(0))
    b = mcr.forward(med, left, spec.forward_run(1))
    both = forward_coefficients(med, spec)
    assert torch.equal(both, a + b)
    # the no-allocation entry point accumulates the same way
    import ctypes as C
    from dataclasses import replace
    c = a.clone()
    run = replace(spec.forward_run(1), accumulate=True)
    rc = mcr.load().mc_forward_noalloc(C.byref(med.c()), C.byref(left.c()), C.byref(run.c()),
                                       C.c_void_p(c.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(c, both)
