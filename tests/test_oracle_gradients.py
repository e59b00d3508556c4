"""Pins of the oracle's functional gradients (Sec. 5, Eqs. 22, 26, 28) and of the adjoint model.

* Quadrature: the closed forms of Eqs. 22 and 26 equal the angular integrals of the radiances
  rebuilt from their Fourier series (Eq. 8), with the phase function of Eq. 6 in closed form.
* Finite differences with common random numbers (CRN): the adjoint gradient (forward run +
  adjoint run from q* = mu_a (H^meas - H), Sec. 6) equals d eps / d mu on tiny grids.  With
  absorption weighting the trajectories do not depend on mu_a, so the CRN difference quotient in
  mu_a is smooth and the check is per pixel and tight; in mu_s it is statistical over seeds.
* A planted mistake (adjoint tallied at theta instead of theta + pi) fails the mu_s check.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import RunParams
from oracle import functionals as F


def _series(coeff, th):
    """phi(theta) = a_0/(2 pi) + (1/pi) sum (a_n cos n theta + b_n sin n theta)  (Eq. 8)."""
    K = (coeff.shape[0] - 1) // 2
    out = np.full(th.shape, coeff[0] / (2 * math.pi))
    for n in range(1, K + 1):
        out = out + (coeff[2 * n - 1] * np.cos(n * th) + coeff[2 * n] * np.sin(n * th)) / math.pi
    return out


@pytest.mark.parametrize("g", [0.3, 0.9])
def test_gradient_integrals_by_quadrature(g):
    """int phi phi* = Eq. 22's sum; int int phi* P phi = Eq. 26; their difference = Eq. 28."""
    rng = np.random.default_rng(17)
    K, npx = 7, 5
    c = rng.normal(size=(2 * K + 1, npx)) / (1 + np.arange(2 * K + 1))[:, None]
    cs = rng.normal(size=(2 * K + 1, npx)) / (1 + np.arange(2 * K + 1))[:, None]
    M = 2048
    th = 2 * math.pi * np.arange(M) / M
    w = 2 * math.pi / M
    P = oracle.hg_phase(g, th)  # P(theta_k - theta_0): circulant kernel on the uniform grid
    for i in range(npx):
        phi = _series(c[:, i], th)
        phs = _series(cs[:, i], th)
        ga = np.sum(phi * phs) * w
        # int phi*(theta) [int P(theta - theta') phi(theta') dtheta'] dtheta  (circular convolution)
        conv = np.real(np.fft.ifft(np.fft.fft(P) * np.fft.fft(phi))) * w
        sc = np.sum(phs * conv) * w
        assert abs(F.G_a(c[:, i:i + 1], cs[:, i:i + 1])[0] - ga) < 1e-9 * (1 + abs(ga))
        assert abs(F.scatter_term(c[:, i:i + 1], cs[:, i:i + 1], g)[0] - sc) < 1e-9 * (1 + abs(sc))
        assert abs(F.G_s(c[:, i:i + 1], cs[:, i:i + 1], g)[0] - (ga - sc)) < 1e-9 * (1 + abs(ga))


def test_paper_forms_equal_general_forms():
    """Eq. 22 / Eq. 28 per unit area times A equal dL/dmu for L = eps, v = -A (H^meas - H)."""
    rng = np.random.default_rng(2)
    K, nz, nx, dx, g = 4, 3, 5, 0.07, 0.8
    c = rng.normal(size=(2 * K + 1, nz, nx))
    cs = rng.normal(size=(2 * K + 1, nz, nx))
    mua = rng.uniform(0.01, 0.2, (nz, nx))
    Hm = rng.uniform(0, 1, (nz, nx))
    v = F.dL_dH_eps(Hm, F.absorbed_energy(mua, c), dx)
    da, ds = F.dL_dmu(c, cs, v, dx, g)
    assert np.allclose(da, dx * dx * F.grad_mua_paper(c, cs, mua, Hm), rtol=1e-13, atol=1e-15)
    assert np.allclose(ds, dx * dx * F.grad_mus_paper(c, cs, g), rtol=1e-13, atol=1e-15)
    q = F.adjoint_source(mua, v, dx)
    assert np.allclose(q, F.adjoint_source_paper(mua, Hm, F.absorbed_energy(mua, c)), rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------- CRN finite differences
def _problem(n, L=0.6):
    dx = L / n
    c = (np.arange(n) + 0.5) * dx
    X, Z = np.meshgrid(c, c)
    mua = 0.15 + 0.1 * np.sin(3 * X) * np.cos(2 * Z)
    mus = 3.0 + 1.0 * np.cos(4 * X + Z)
    mua_true = mua * (1 + 2 * np.exp(-((X - 0.35) ** 2 + (Z - 0.3) ** 2) / 0.02))
    src = dict(kind=oracle.LINE, x0=0.0, z0=0.0, x1=L, z1=0.0, dir_x=0.0, dir_z=1.0)
    return dx, X, Z, mua, mus, mua_true, src


def _adjoint_gradient(mua, mus, dx, g, src, Hm, K, n_fwd, n_adj, seed, flip=True):
    Fc = oracle.forward(mua, mus, dx, g, src, RunParams(K=K, n_packets=n_fwd, seed=seed)).coeff
    v = F.dL_dH_eps(Hm, F.absorbed_energy(mua, Fc), dx)
    q = F.adjoint_source(mua, v, dx).astype(np.float32)
    A = oracle.volume(mua, mus, dx, g, q, RunParams(K=K, n_packets=n_adj, seed=seed + 1000, stream_id=1),
                      adjoint=flip).coeff
    return F.dL_dmu(Fc, A, v, dx, g)


def _eps(mua, mus, dx, g, src, Hm, n, seed):
    c = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=n, seed=seed)).coeff
    return F.error_functional(Hm, F.absorbed_energy(mua, c), dx)


def test_mua_gradient_matches_crn_finite_differences():
    """Per pixel: adjoint d eps/d mu_a (Eq. 22 x A) vs central CRN differences, 6x6 grid."""
    g = 0.5
    dx, X, Z, mua, mus, mua_true, src = _problem(6)
    Hm = F.absorbed_energy(mua_true, oracle.forward(mua_true, mus, dx, g, src,
                                                    RunParams(K=0, n_packets=1_000_000, seed=99)).coeff)
    n = 200_000
    ga, _ = _adjoint_gradient(mua, mus, dx, g, src, Hm, 12, n, 1_000_000, seed=1)
    fd = np.zeros_like(mua)
    h = 1e-4
    for idx in np.ndindex(mua.shape):
        e = np.zeros_like(mua)
        e[idx] = h
        fd[idx] = (_eps(mua + e, mus, dx, g, src, Hm, n, 1) - _eps(mua - e, mus, dx, g, src, Hm, n, 1)) / (2 * h)
    scale = np.max(np.abs(fd))
    # the remainder is the pixel-mean product (discretisation) and the adjoint run's noise
    assert np.max(np.abs(ga - fd)) < 3e-3 * scale
    assert np.corrcoef(ga.ravel(), fd.ravel())[0, 1] > 0.9999


REGIONS = [(0.2, 0.4, 0.0, 0.2), (0.0, 0.2, 0.2, 0.4), (0.4, 0.6, 0.4, 0.6), (0.2, 0.4, 0.2, 0.4)]


def _mus_block_study(flip, seeds):
    g = 0.5
    dx, X, Z, mua, mus, mua_true, src = _problem(12)
    Hm = F.absorbed_energy(mua_true, oracle.forward(mua_true, mus, dx, g, src,
                                                    RunParams(K=0, n_packets=2_000_000, seed=99)).coeff)
    n = 200_000
    rows = []
    for seed in seeds:
        _, gs = _adjoint_gradient(mua, mus, dx, g, src, Hm, 32, n, 1_000_000, seed=seed, flip=flip)
        row = []
        for (x0, x1, z0, z1) in REGIONS:
            m = ((X > x0) & (X < x1) & (Z > z0) & (Z < z1)).astype(float)
            h = 0.05  # relative change of mu_s over the block
            fd = (_eps(mua, mus * (1 + h * m), dx, g, src, Hm, n, seed)
                  - _eps(mua, mus * (1 - h * m), dx, g, src, Hm, n, seed)) / (2 * h)
            row.append((fd, float(np.sum(gs * mus * m))))  # directional derivative along mu_s * block
        rows.append(row)
    r = np.array(rows)
    d = r[:, :, 1] - r[:, :, 0]
    return r, d.mean(0), d.std(0, ddof=1) / math.sqrt(len(seeds))


@pytest.mark.slow
def test_mus_gradient_matches_crn_finite_differences():
    """Block directional derivatives in mu_s: adjoint (Eq. 28 x A) vs CRN differences agree within
    4 standard errors over 4 seeds plus a discretisation budget of 5% of the largest block
    derivative (the gradient uses products of pixel means, not pixel means of products)."""
    r, mean, se = _mus_block_study(True, (1, 3, 5, 7))
    size = np.abs(r[:, :, 0].mean(0))
    assert np.all(np.abs(mean) < 4 * se + 0.05 * size.max()), (mean, se, size)
    assert np.all(np.abs(mean) < 0.15 * size + 0.05 * size.max()), (mean, size)


@pytest.mark.slow
def test_planted_missing_adjoint_flip_fails_fd():
    """Tallying the adjoint run at theta (no theta + pi) breaks the mu_s gradient: the block
    derivative next to the collimated source then misses the CRN difference by many sigma."""
    r, mean, se = _mus_block_study(False, (1, 3))
    size = np.abs(r[:, :, 0].mean(0))
    assert np.abs(mean[0]) > 0.2 * size[0]
