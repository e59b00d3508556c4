"""Pins of the 3D oracle (the spherical-harmonic extension Sec. 3.1 names): its basis, its
Henyey-Greenstein sampler, transport and bookkeeping, the adjoint's turn of the tally, and its
functional gradients against finite differences with common random numbers (CPU only)."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, roots_legendre

import oracle
from oracle import RunParams
from oracle import functionals as F


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_spherical_harmonics_are_orthonormal_and_satisfy_the_addition_theorem():
    L = 6
    x, wx = roots_legendre(40)
    nphi = 80
    phi = 2 * math.pi * np.arange(nphi) / nphi
    C = (L + 1) ** 2
    G = np.zeros((C, C))
    for ct, w in zip(x, wx):
        st = math.sqrt(1 - ct * ct)
        for ph in phi:
            Y = oracle.sh3(L, st * math.cos(ph), st * math.sin(ph), ct)
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    assert np.allclose(G, np.eye(C), atol=1e-12)
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = _unit(rng.normal(size=3)), _unit(rng.normal(size=3))
        Ya, Yb = oracle.sh3(L, *a), oracle.sh3(L, *b)
        for l in range(L + 1):
            s = sum(Ya[l * l + l + m] * Yb[l * l + l + m] for m in range(-l, l + 1))
            assert abs(s - (2 * l + 1) / (4 * math.pi) * eval_legendre(l, float(a @ b))) < 1e-12
    # Y_lm(-s) = (-1)^l Y_lm(s): the adjoint's turn of the tally
    s = _unit([0.3, -0.7, 0.2])
    Yp, Ym = oracle.sh3(L, *s), oracle.sh3(L, *(-s))
    for l in range(L + 1):
        for m in range(-l, l + 1):
            assert abs(Ym[l * l + l + m] - (-1) ** l * Yp[l * l + l + m]) < 1e-14


@pytest.mark.parametrize("g", [0.0, 0.5, 0.9, -0.3])
def test_hg3_sampler_has_the_phase_function_moments(g):
    """E[P_l(cos)] = g^l for the 3D Henyey-Greenstein phase function, by quadrature over u of the
    inverse-CDF sampler (no sampling noise)."""
    u, w = roots_legendre(400)
    u, w = 0.5 * (u + 1), 0.5 * w
    c = np.array([oracle.hg3_cos(g, ui) for ui in u])
    for l in range(1, 9):
        assert abs(float(np.sum(w * eval_legendre(l, c))) - g ** l) < 1e-9, l


def _chords(x0, d, nx, ny, nz, dx):
    """Voxels and path lengths of the ray x0 + s d through the grid (independent: sort all face
    crossings)."""
    ts = [0.0]
    for k, n in enumerate((nx, ny, nz)):
        if d[k] != 0:
            for i in range(n + 1):
                t = (i * dx - x0[k]) / d[k]
                if t > 0:
                    ts.append(t)
    ts = sorted(set(ts))
    out = []
    for a, b in zip(ts, ts[1:]):
        mid = x0 + 0.5 * (a + b) * d
        idx = np.floor(mid / dx).astype(int)
        if np.all(idx >= 0) and idx[0] < nx and idx[1] < ny and idx[2] < nz:
            out.append(((idx[2], idx[1], idx[0]), b - a))
        elif out:
            break
    return out


def test_beer_lambert_3d_closed_form():
    """mu_s = 0: every packet follows the same oblique ray; voxel coefficients are
    t Y_lm(s0) / V with t = exp(-absorption so far) (1 - exp(-mu_a l)) / mu_a (1e-12)."""
    nz, ny, nx, dx, L = 5, 4, 6, 0.2, 3
    rng = np.random.default_rng(4)
    mua = rng.uniform(0.1, 2.0, (nz, ny, nx))
    mus = np.zeros((nz, ny, nx))
    d = _unit([0.35, -0.2, 1.0])
    x0 = np.array([0.33, 0.61, 0.0])
    src = dict(kind=oracle.PENCIL, x0=x0[0], y0=x0[1], z0=0.0, dir_x=d[0], dir_y=d[1], dir_z=d[2])
    r = oracle.forward3(mua, mus, dx, 0.5, src, RunParams(K=L, n_packets=5, n_threads=1))
    want = np.zeros_like(r.coeff)
    Y = oracle.sh3(L, *d)
    T = 1.0
    for (iz, iy, ix), l in _chords(x0, d, nx, ny, nz, dx):
        a = mua[iz, iy, ix]
        want[:, iz, iy, ix] += T * (1 - math.exp(-a * l)) / a * Y / dx ** 3
        T *= math.exp(-a * l)
    assert np.allclose(r.coeff, want, rtol=1e-12, atol=1e-14)


def _hetero3(nz, ny, nx, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.05, 0.8, (nz, ny, nx)), rng.uniform(0.5, 6.0, (nz, ny, nx))


def test_energy_conservation_3d():
    """launched + roulette gain = absorbed + escaped + killed, and the absorbed weight equals
    sum_v mu_a,v Phi_v V N_p (Phi = sqrt(4 pi) c_00)."""
    nz, ny, nx, dx = 6, 5, 7, 0.15
    mua, mus = _hetero3(nz, ny, nx, 5)
    src = dict(kind=oracle.ISO_POINT, x0=0.51, y0=0.4, z0=0.47)
    N = 20000
    r = oracle.forward3(mua, mus, dx, 0.7, src, RunParams(K=2, n_packets=N, seed=9, w_threshold=0.9,
                                                          roulette_p=0.5))
    st = r.stats
    assert abs(st["launched_w"] + st["rr_net_w"] - st["absorbed_w"] - st["escaped_w"] - st["killed_w"]) < 1e-11 * N
    absorbed = float(np.sum(mua * F.fluence3(r.coeff))) * dx ** 3 * N
    assert abs(absorbed - st["absorbed_w"]) < 1e-9 * st["absorbed_w"]
    assert st["rr_kill"] > 0 and st["rr_survive"] > 0


def test_reciprocity_case1_voxel_sources_3d():
    """Case 1 (Eqs. 14, 17) in 3D: unit isotropic sources uniform over voxel s and voxel d give
    Phi_s(d) = Phi_d(s) in a heterogeneous scattering medium."""
    nz, ny, nx, dx = 8, 7, 9, 0.1
    mua, mus = _hetero3(nz, ny, nx, 11)
    mus = mus * 1.5
    for k, (s, d) in enumerate([((1, 2, 3), (6, 4, 6)), ((4, 0, 1), (4, 6, 7))]):
        def unit(p):
            q = np.zeros((nz, ny, nx), np.float32)
            q[p] = 1.0 / (4 * math.pi * dx ** 3)
            return q
        run = RunParams(K=0, n_packets=300000, seed=100 + k)
        fs = oracle.volume3(mua, mus, dx, 0.6, unit(s), run, adjoint=False, with_variance=True)
        fd = oracle.volume3(mua, mus, dx, 0.6, unit(d), run, adjoint=True, with_variance=True)
        assert abs(fs.source_strength - 1.0) < 1e-6
        a, b = F.fluence3(fs.coeff)[d], F.fluence3(fd.coeff)[s]
        sig = math.sqrt(4 * math.pi) * math.sqrt(fs.a0_var[d] + fd.a0_var[s]) / math.sqrt(4 * math.pi)
        assert abs(a - b) < 5 * sig, (s, d, a, b, sig)
        assert a > 10 * sig


def test_adjoint_tally_is_turned_by_pi():
    """On the same packets the adjoint run's coefficients are (-1)^l times the forward ones."""
    nz, ny, nx, dx, L = 4, 4, 4, 0.2, 4
    mua, mus = _hetero3(nz, ny, nx, 2)
    q = np.zeros((nz, ny, nx), np.float32)
    q[1, 2, 1] = 1.0
    q[3, 0, 2] = -0.5
    run = RunParams(K=L, n_packets=3000, seed=4, n_threads=1)
    fwd = oracle.volume3(mua, mus, dx, 0.8, q, run, adjoint=False).coeff
    adj = oracle.volume3(mua, mus, dx, 0.8, q, run, adjoint=True).coeff
    for c in range(fwd.shape[0]):
        l = math.isqrt(c)
        assert np.allclose(adj[c], (-1) ** l * fwd[c], rtol=1e-12, atol=1e-15)
    assert np.abs(fwd[1:4]).max() > 0  # the odd channels are not trivially zero


def _problem3(n, L=0.6):
    dx = L / n
    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    mua = 0.15 + 0.1 * np.sin(3 * X) * np.cos(2 * Z) + 0.05 * np.cos(5 * Y)
    mus = 3.0 + 1.0 * np.cos(4 * X + Z - Y)
    mua_true = mua * (1 + 2 * np.exp(-((X - 0.35) ** 2 + (Y - 0.25) ** 2 + (Z - 0.3) ** 2) / 0.02))
    src = dict(kind=oracle.PENCIL, x0=0.5 * L, y0=0.45 * L, z0=0.0, dir_x=0.0, dir_y=0.0, dir_z=1.0)
    return dx, mua, mus, mua_true, src


def _eps3(mua, mus, dx, g, src, Hm, n, seed):
    c = oracle.forward3(mua, mus, dx, g, src, RunParams(K=0, n_packets=n, seed=seed)).coeff
    return F.error_functional3(Hm, F.absorbed_energy3(mua, c), dx)


def _adjoint_gradient3(mua, mus, dx, g, src, Hm, L, n_fwd, n_adj, seed, flip=True):
    Fc = oracle.forward3(mua, mus, dx, g, src, RunParams(K=L, n_packets=n_fwd, seed=seed)).coeff
    v = F.dL_dH_eps3(Hm, F.absorbed_energy3(mua, Fc), dx)
    q = F.adjoint_source3(mua, v, dx).astype(np.float32)
    A = oracle.volume3(mua, mus, dx, g, q, RunParams(K=L, n_packets=n_adj, seed=seed + 1000, stream_id=1),
                       adjoint=flip).coeff
    return F.dL_dmu3(Fc, A, v, dx, g)


def test_mua_gradient_3d_matches_crn_finite_differences():
    """Per voxel: the adjoint gradient d eps / d mu_a = v Phi + V sum_lm c_lm c*_lm against central
    differences with common random numbers (trajectories do not depend on mu_a), 4^3 grid."""
    g = 0.5
    dx, mua, mus, mua_true, src = _problem3(4)
    Hm = F.absorbed_energy3(mua_true, oracle.forward3(mua_true, mus, dx, g, src,
                                                      RunParams(K=0, n_packets=400_000, seed=99)).coeff)
    n = 60_000
    ga, _ = _adjoint_gradient3(mua, mus, dx, g, src, Hm, 6, n, 400_000, seed=1)
    fd = np.zeros_like(mua)
    h = 1e-4
    for idx in np.ndindex(mua.shape):
        e = np.zeros_like(mua)
        e[idx] = h
        fd[idx] = (_eps3(mua + e, mus, dx, g, src, Hm, n, 1) - _eps3(mua - e, mus, dx, g, src, Hm, n, 1)) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(ga - fd)) < 1e-2 * scale, (np.max(np.abs(ga - fd)) / scale)
    assert np.corrcoef(ga.ravel(), fd.ravel())[0, 1] > 0.999


def test_mua_gradient_3d_without_the_turn_fails():
    """The planted mistake (adjoint tallied at s, not -s) misses the CRN differences by > 4 %."""
    g = 0.5
    dx, mua, mus, mua_true, src = _problem3(4)
    Hm = F.absorbed_energy3(mua_true, oracle.forward3(mua_true, mus, dx, g, src,
                                                      RunParams(K=0, n_packets=400_000, seed=99)).coeff)
    n = 60_000
    ga, _ = _adjoint_gradient3(mua, mus, dx, g, src, Hm, 6, n, 400_000, seed=1, flip=False)
    fd = np.zeros_like(mua)
    h = 1e-4
    for idx in np.ndindex(mua.shape):
        e = np.zeros_like(mua)
        e[idx] = h
        fd[idx] = (_eps3(mua + e, mus, dx, g, src, Hm, n, 1) - _eps3(mua - e, mus, dx, g, src, Hm, n, 1)) / (2 * h)
    assert np.max(np.abs(ga - fd)) > 4e-2 * np.max(np.abs(fd))


def test_mus_gradient_3d_matches_crn_finite_differences():
    """Block directional derivatives in mu_s, d eps = sum_v V sum_lm (1 - g^l) c_lm c*_lm dmu_s, on an
    8^3 grid lit by isotropic sources spread over its top layer (a diffuse field, so the truncation
    at l = 6 is immaterial): within 4 standard errors over 4 seeds plus 10 %.  (On a 4^3 grid the
    products of voxel means differ from the means of products by ~25 %: a discretisation effect that
    the refinement removes.)  Without the turn of the adjoint tally the sign is wrong."""
    g, n = 0.5, 8
    dx, mua, mus, mua_true, _ = _problem3(n)
    qf = np.zeros(mua.shape, np.float32)
    qf[0] = 1.0

    def fwd(mua_, mus_, L, npk, seed):
        return oracle.volume3(mua_, mus_, dx, g, qf, RunParams(K=L, n_packets=npk, seed=seed), adjoint=False).coeff

    Hm = F.absorbed_energy3(mua_true, fwd(mua_true, mus, 0, 400_000, 99))

    def eps(mus_, seed):
        return F.error_functional3(Hm, F.absorbed_energy3(mua, fwd(mua, mus_, 0, 100_000, seed)), dx)

    def grad(seed, flip=True):
        Fc = fwd(mua, mus, 6, 100_000, seed)
        v = F.dL_dH_eps3(Hm, F.absorbed_energy3(mua, Fc), dx)
        q = F.adjoint_source3(mua, v, dx).astype(np.float32)
        A = oracle.volume3(mua, mus, dx, g, q, RunParams(K=6, n_packets=600_000, seed=seed + 1000, stream_id=1),
                           adjoint=flip).coeff
        return F.dL_dmu3(Fc, A, v, dx, g)[1]

    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    seeds = (1, 3, 5, 7)
    h = 0.05
    fd_top = None
    for m in ((Z < 0.3).astype(float), (X < 0.3).astype(float)):
        fd = np.array([(eps(mus * (1 + h * m), s) - eps(mus * (1 - h * m), s)) / (2 * h) for s in seeds])
        ad = np.array([float(np.sum(grad(s) * mus * m)) for s in seeds])
        d = ad - fd
        se = d.std(ddof=1) / math.sqrt(len(seeds))
        assert abs(d.mean()) < 4 * se + 0.1 * abs(fd.mean()), (fd.mean(), ad.mean(), se)
        fd_top = fd.mean() if fd_top is None else fd_top
    wrong = float(np.sum(grad(1, flip=False) * mus * (Z < 0.3)))
    assert wrong * fd_top < 0 or abs(wrong - fd_top) > 0.5 * abs(fd_top), (wrong, fd_top)
