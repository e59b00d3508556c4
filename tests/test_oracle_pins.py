"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form
(Beer-Lambert, uncollided fluence, HG moments), exact bookkeeping, the adjoint
transport equation, or an independent numerical construction (ray-pixel chords,
quadrature).  The finite-difference gradient pins live in test_oracle_gradients.py.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from oracle import RunParams


# ----------------------------------------------------------------------------- RNG
def test_philox_uniform_and_independent():
    """Philox4x32-10 words are uniform, bit-balanced and uncorrelated across counters."""
    key = (0x12345678, 0x9ABCDEF0)
    words = np.array([oracle.philox4x32_10((p, 0, e, 0), key) for p in range(2048) for e in range(4)],
                     dtype=np.uint64).reshape(2048, 4, 4)
    u = oracle.u01(words).ravel()
    # uniformity (KS) and bit balance of all 32 bits
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    bits = np.array([(words.ravel() >> np.uint64(b)) & np.uint64(1) for b in range(32)], dtype=np.float64)
    assert np.all(np.abs(bits.mean(axis=1) - 0.5) < 5 * 0.5 / math.sqrt(words.size))
    # neighbouring packets / events are uncorrelated
    up = oracle.u01(words[:, 0, 0])
    for other in (oracle.u01(words[:, 1, 0]), oracle.u01(np.roll(words[:, 0, 0], 1)), oracle.u01(words[:, 0, 1])):
        assert abs(np.corrcoef(up, other)[0, 1]) < 5 / math.sqrt(up.size)
    # counter and key both matter
    assert not np.array_equal(oracle.philox4x32_10((0, 0, 0, 0), (0, 0)), oracle.philox4x32_10((1, 0, 0, 0), (0, 0)))
    assert not np.array_equal(oracle.philox4x32_10((0, 0, 0, 0), (0, 0)), oracle.philox4x32_10((0, 0, 0, 0), (1, 0)))


def _philox_kat():
    """The published Philox4x32-10 known-answer vectors (tests/golden/philox4x32_10_kat.txt)."""
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


def test_philox_known_answers():
    """The oracle's Philox4x32-10 reproduces the generator's published known answers (zero counter
    and key, all-ones counter and key, and the pi-digits vector): a swapped output word, a wrong
    multiplier or Weyl constant, or a wrong round count fails all three."""
    kat = _philox_kat()
    assert len(kat) == 3
    for ctr, key, want in kat:
        assert tuple(int(v) for v in oracle.philox4x32_10(ctr, key)) == want


def test_uniform_map_exact_in_fp32():
    """u = ((x>>9)+1/2) 2^-23 is exactly representable in FP32 and lies strictly inside (0, 1)."""
    x = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1, 0xDEADBEEF], dtype=np.uint64)
    u = oracle.u01(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)


# ------------------------------------------------------------------- HG (Eqs. 6, 7, 24)
@pytest.mark.parametrize("g", [0.0, 0.5, 0.8, 0.9, -0.3])
def test_hg_sampler_circular_moments(g):
    """E[cos n theta_s] = g^n and E[sin n theta_s] = 0 for the sampler of Eq. 7.

    These are the Fourier coefficients of the phase function (Eq. 24); the expectation over
    U ~ U(0,1) is evaluated by the midpoint rule, which converges spectrally for this smooth
    periodic integrand.
    """
    n_u = 1 << 15
    u = (np.arange(n_u) + 0.5) / n_u
    th = oracle.hg_angle(g, u)
    for n in range(1, 9):
        assert abs(np.mean(np.cos(n * th)) - g ** n) < 1e-9
        assert abs(np.mean(np.sin(n * th))) < 1e-9


@pytest.mark.parametrize("g", [0.0, 0.7, 0.9])
def test_hg_sampler_distribution_matches_phase_function(g):
    """The angles of Eq. 7 are distributed as the phase function of Eq. 6 (KS on the exact CDF)."""
    n_u = 4000
    u = (np.arange(n_u) + 0.5) / n_u
    th = oracle.hg_angle(g, u)

    def cdf(x):
        return integrate.quad(lambda t: oracle.hg_phase(g, t)[0], -math.pi, x, limit=200)[0]

    xs = np.linspace(-math.pi + 1e-3, math.pi - 1e-3, 41)
    emp = np.array([np.mean(th <= x) for x in xs])
    ref = np.array([cdf(x) for x in xs])
    assert np.max(np.abs(emp - ref)) < 2.0 / n_u


@pytest.mark.parametrize("g", [0.0, 0.6, 0.9])
def test_hg_phase_normalised_and_fourier_series(g):
    """Eq. 6 integrates to 1 and has the cosine series of Eq. 24 (coefficients g^l / pi)."""
    th = np.linspace(-math.pi, math.pi, 4097)[:-1]
    P = oracle.hg_phase(g, th)
    w = 2 * math.pi / th.size
    assert abs(P.sum() * w - 1.0) < 1e-10
    for l in range(1, 6):
        assert abs((P * np.cos(l * th)).sum() * w - g ** l) < 1e-10


# --------------------------------------------------------------- Beer-Lambert (exact)
def _chords(x0, z0, sx, sz, nx, nz, dx):
    """Ray-pixel chord lengths by sorting all grid-line crossings (independent of the DDA)."""
    W, D = nx * dx, nz * dx
    ts = [0.0]
    for k in range(nx + 1):
        if sx != 0:
            t = (k * dx - x0) / sx
            if t > 0:
                ts.append(t)
    for k in range(nz + 1):
        if sz != 0:
            t = (k * dx - z0) / sz
            if t > 0:
                ts.append(t)
    ts = np.unique(np.array(ts))
    out = []
    for a, b in zip(ts[:-1], ts[1:]):
        m = 0.5 * (a + b)
        xm, zm = x0 + m * sx, z0 + m * sz
        if not (0 <= xm < W and 0 <= zm < D):
            break
        out.append((int(zm // dx), int(xm // dx), b - a))
    return out


@pytest.mark.parametrize("angle_deg", [0.0, 23.0, -61.0])
def test_beer_lambert_closed_form(angle_deg):
    """mu_s = 0: every packet follows one ray; a_0 is the attenuated track length per area.

    a_0,i = exp(-sum_prev mu_a l) (1 - exp(-mu_a,i l_i)) / (mu_a,i A), a_n = a_0 cos(n theta),
    b_n = a_0 sin(n theta), independent of N_p (Sec. 3 deposit with absorption weighting).
    """
    rng = np.random.default_rng(3)
    nz, nx, dx = 9, 11, 0.3
    mua = rng.uniform(0.05, 1.5, (nz, nx))
    mua[4, 5] = 0.0  # the t = W l branch
    mus = np.zeros((nz, nx))
    th = math.radians(angle_deg)
    sx, sz = math.sin(th), math.cos(th)
    x0, z0 = 1.73, 0.0
    K = 5
    r = oracle.forward(mua, mus, dx, 0.5, dict(kind=oracle.PENCIL, x0=x0, z0=z0, dir_x=sx, dir_z=sz),
                       RunParams(K=K, n_packets=7, n_threads=2))
    expect = np.zeros((2 * K + 1, nz, nx))
    W = 1.0
    for iz, ix, l in _chords(x0, z0, sx, sz, nx, nz, dx):
        m = mua[iz, ix]
        t = W * (1 - math.exp(-m * l)) / m if m > 0 else W * l
        W *= math.exp(-m * l)
        expect[0, iz, ix] += t / (dx * dx)
    for n in range(1, K + 1):
        expect[2 * n - 1] = expect[0] * math.cos(n * th)
        expect[2 * n] = expect[0] * math.sin(n * th)
    assert np.max(np.abs(r.coeff - expect)) <= 1e-12 * np.max(expect[0])
    assert r.stats["escapes"] == 7


def test_pencil_unit_fluence_without_absorption():
    """mu_a = mu_s = 0: a straight beam gives a_0 = 1/dx in every pixel of its column."""
    nz, nx, dx = 6, 5, 0.2
    z = np.zeros((nz, nx))
    r = oracle.forward(z, z, dx, 0.0, dict(kind=oracle.PENCIL, x0=0.5, z0=0.0, dir_x=0.0, dir_z=1.0),
                       RunParams(K=2, n_packets=3, n_threads=1))
    col = np.zeros((nz, nx))
    col[:, 2] = 1.0 / dx
    assert np.allclose(r.coeff[0], col, rtol=1e-13, atol=1e-13)
    assert np.allclose(r.coeff[1], col, rtol=1e-13, atol=1e-13)  # a_1 = a_0 cos 0
    assert np.allclose(r.coeff[2], 0.0, atol=1e-13)              # b_1 = a_0 sin 0


# ------------------------------------------------------------ energy bookkeeping (exact)
def _hetero(nz, nx, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.02, 0.6, (nz, nx)), rng.uniform(0.5, 8.0, (nz, nx))


@pytest.mark.parametrize("mode", ["line", "adjoint"])
def test_energy_conservation(mode):
    """launched + roulette gain = absorbed + escaped + killed, and the absorbed weight equals
    sum_i mu_a,i a_0,i A N_p / S (the tally of track weights times mu_a)."""
    nz, nx, dx = 12, 10, 0.15
    mua, mus = _hetero(nz, nx, 5)
    run = RunParams(K=3, n_packets=20000, seed=9, w_threshold=0.95, roulette_p=0.5, max_scatter=3)
    if mode == "line":
        r = oracle.forward(mua, mus, dx, 0.7, dict(kind=oracle.LINE, x0=0.0, z0=0.0, x1=nx * dx, z1=0.0,
                                                   dir_x=0.0, dir_z=1.0), run)
    else:
        q = np.random.default_rng(1).normal(size=(nz, nx)).astype(np.float32)
        r = oracle.adjoint(mua, mus, dx, 0.7, q, run)
    st = r.stats
    assert st["rr_kill"] > 0 and st["rr_survive"] > 0 and st["scatter_limit"] > 0
    lhs = st["launched_w"] + st["rr_net_w"]
    rhs = st["absorbed_w"] + st["escaped_w"] + st["killed_w"]
    assert abs(lhs - rhs) <= 1e-11 * run.n_packets
    from_tally = float(np.sum(mua * r.coeff[0])) * dx * dx * run.n_packets / r.source_strength
    assert abs(from_tally - st["absorbed_w"]) <= 1e-11 * run.n_packets


def test_event_limit_ends_packets():
    nz, nx, dx = 8, 8, 0.5
    mua, mus = np.full((nz, nx), 0.001), np.full((nz, nx), 20.0)
    r = oracle.forward(mua, mus, dx, 0.0, dict(kind=oracle.ISO_POINT, x0=2.0, z0=2.0),
                       RunParams(K=1, n_packets=50, max_events=5, n_threads=1))
    assert r.stats["event_limit"] == 50 and r.stats["flights"] == 250


# --------------------------------------------------------- uncollided fluence (closed form)
def _uncollided_pixel_means(nz, nx, dx, xs, zs, mut, sub=24):
    """Pixel means of exp(-mu_t r) cos(n phi)/(2 pi r) (phi = atan2(x-xs, z-zs)), n = 0, 1 (a and b)."""
    o = (np.arange(sub) + 0.5) / sub * dx
    out = np.zeros((3, nz, nx))
    for iz in range(nz):
        for ix in range(nx):
            X, Z = np.meshgrid(ix * dx + o, iz * dx + o)
            r = np.hypot(X - xs, Z - zs)
            phi = np.arctan2(X - xs, Z - zs)
            f = np.exp(-mut * r) / (2 * math.pi * r)
            out[0, iz, ix] = f.mean()
            out[1, iz, ix] = (f * np.cos(phi)).mean()
            out[2, iz, ix] = (f * np.sin(phi)).mean()
    return out


def test_uncollided_fluence_point_source():
    """Isotropic point source, packets ended at their first collision: the tally is the
    uncollided radiance exp(-(mu_a+mu_s) r)/(2 pi r) along the outward ray, so
    a_0 = pixel mean of that, a_1 + i b_1 = pixel mean times exp(i phi)."""
    nz, nx, dx = 14, 14, 0.1
    mua, mus = 0.4, 2.0
    xs, zs = 0.7, 0.7
    r = oracle.forward(np.full((nz, nx), mua), np.full((nz, nx), mus), dx, 0.9,
                       dict(kind=oracle.ISO_POINT, x0=xs, z0=zs),
                       RunParams(K=1, n_packets=400000, seed=2, max_scatter=0), with_variance=True)
    ref = _uncollided_pixel_means(nz, nx, dx, xs, zs, mua + mus)
    far = np.ones((nz, nx), bool)
    far[5:9, 5:9] = False  # the four pixels touching the source and their ring: singular pixel means
    sig = np.sqrt(r.a0_var)
    z0 = (r.coeff[0] - ref[0])[far] / sig[far]
    assert np.max(np.abs(z0)) < 5.0
    assert abs(np.mean(z0)) < 4.0 / math.sqrt(z0.size)
    # harmonics: |a_n| <= a_0 per packet, so a_0's sigma bounds theirs
    for c in (1, 2):
        zc = (r.coeff[c] - ref[c])[far] / sig[far]
        assert np.max(np.abs(zc)) < 5.0


def _ring_sums(field, R, edges):
    return np.array([field[(R >= lo) & (R < hi)].sum() for lo, hi in zip(edges[:-1], edges[1:])])


def test_diffusion_far_field_fluence_and_flux():
    """Deep in a scattering medium (mu_a << mu_s') the oracle's a_0 follows the 2D diffusion
    Green's function Phi = K_0(kappa r)/(2 pi D), D = 1/(2(mu_a + mu_s(1-g))), kappa^2 = mu_a/D,
    and its first harmonics follow Fick's law: with Eq. 8, phi = a_0/(2 pi) + (a_1 cos + b_1 sin)/pi,
    so (b_1, a_1) = J = kappa K_1(kappa r)/(2 pi) r_hat (radial, no tangential part).  A 5 %
    budget covers diffusion theory's own error at mu_a/mu_s' = 0.04 and r >= 3/mu_s'."""
    from scipy.special import k0, k1
    n, dx = 60, 0.2
    mua, mus, g = 0.2, 10.0, 0.5
    xs = zs = n * dx / 2
    r = oracle.forward(np.full((n, n), mua), np.full((n, n), mus), dx, g, dict(kind=oracle.ISO_POINT, x0=xs, z0=zs),
                       RunParams(K=2, n_packets=20000, seed=3), with_variance=True)
    D = 1 / (2 * (mua + mus * (1 - g)))
    kappa = math.sqrt(mua / D)
    sub = 8
    o = (np.arange(sub) + 0.5) / sub * dx
    phi, flux = np.zeros((n, n)), np.zeros((n, n))
    for iz in range(n):
        for ix in range(n):
            X, Z = np.meshgrid(ix * dx + o, iz * dx + o)
            rr = np.hypot(X - xs, Z - zs)
            phi[iz, ix] = (k0(kappa * rr) / (2 * math.pi * D)).mean()
            flux[iz, ix] = (kappa * k1(kappa * rr) / (2 * math.pi)).mean()
    c = (np.arange(n) + 0.5) * dx
    X, Z = np.meshgrid(c, c)
    R = np.hypot(X - xs, Z - zs)
    edges = np.arange(0.6, 3.01, 0.4)
    ratio = _ring_sums(r.coeff[0], R, edges) / _ring_sums(phi, R, edges)
    assert np.all(np.abs(ratio - 1) < 0.05), ratio
    jr = (r.coeff[2] * (X - xs) + r.coeff[1] * (Z - zs)) / R
    jt = (r.coeff[2] * (Z - zs) - r.coeff[1] * (X - xs)) / R
    jr_ring = _ring_sums(jr, R, edges)
    assert np.all(np.abs(jr_ring / _ring_sums(flux, R, edges) - 1) < 0.05)
    assert np.all(np.abs(_ring_sums(jt, R, edges) / jr_ring) < 0.05)


def test_mirror_symmetry_of_harmonics():
    """A medium and a source symmetric under x -> L - x give mirror-symmetric radiance: theta ->
    -theta, so a_n(x) = a_n(L - x) and b_n(x) = -b_n(L - x) (statistically; |a_n|, |b_n| <= a_0
    per deposit, so a_0's standard error bounds theirs)."""
    nz, nx, dx = 24, 31, 0.1  # odd width: the pencil runs down the middle of column 15
    mua, mus = _hetero(nz, nx, 21)
    mua = 0.5 * (mua + mua[:, ::-1])
    mus = 0.5 * (mus + mus[:, ::-1])
    r = oracle.forward(mua, mus, dx, 0.7, dict(kind=oracle.PENCIL, x0=nx * dx / 2, z0=0.0, dir_x=0.0, dir_z=1.0),
                       RunParams(K=3, n_packets=100000, seed=9), with_variance=True)
    sig = np.sqrt(r.a0_var + r.a0_var[:, ::-1])
    use = r.coeff[0] > 0.02 * r.coeff[0].max()
    zs_ = []
    for c in range(7):
        sign = 1.0 if c == 0 or c % 2 == 1 else -1.0  # channel 2n-1 = a_n (even), 2n = b_n (odd)
        d = (r.coeff[c] - sign * r.coeff[c][:, ::-1])[use] / sig[use]
        assert np.max(np.abs(d)) < 6.0, c
        zs_.append(d)
    assert abs(np.mean(np.concatenate(zs_))) < 0.1
    # b_n themselves are far from zero off the axis: the test is not vacuous
    assert np.abs(r.coeff[2][use]).max() > 20 * sig[use].max()


# ------------------------------------------------------------ reciprocity (Eqs. 13, 17)
def test_reciprocity_case1_pixel_sources():
    """Case 1 (Eqs. 14, 17): isotropic unit sources uniform over pixel s and pixel d give
    Phi_s(d) = Phi_d(s) in a heterogeneous scattering medium."""
    nz, nx, dx = 16, 16, 0.1
    mua, mus = _hetero(nz, nx, 11)
    g = 0.6
    pairs = [((3, 4), (11, 12)), ((8, 2), (8, 13)), ((1, 7), (14, 7))]
    for k, (s, d) in enumerate(pairs):
        def unit(p):
            q = np.zeros((nz, nx), np.float32)
            q[p] = 1.0 / (2 * math.pi * dx * dx)
            return q
        run = RunParams(K=0, n_packets=200000, seed=100 + k)
        fs = oracle.volume(mua, mus, dx, g, unit(s), run, adjoint=False, with_variance=True)
        fd = oracle.volume(mua, mus, dx, g, unit(d), run, adjoint=True, with_variance=True)
        assert abs(fs.source_strength - 1.0) < 1e-7  # q is stored in FP32
        a, b = fs.coeff[0][d], fd.coeff[0][s]
        sig = math.sqrt(fs.a0_var[d] + fd.a0_var[s])
        assert abs(a - b) < 5 * sig, (s, d, a, b, sig)
        assert a > 10 * sig


def test_point_source_vs_volume_source_normalisation():
    """A unit isotropic point source at the centre of pixel s and a unit volumetric adjoint
    source in a far pixel d see the same fluence at each other's pixel (Eq. 17); this fixes the
    volumetric strength S = 2 pi A sum|q*| against the forward normalisation."""
    nz, nx, dx = 20, 20, 0.1
    mua, mus = np.full((nz, nx), 0.3), np.full((nz, nx), 4.0)
    s, d = (5, 5), (14, 13)
    fwd = oracle.forward(mua, mus, dx, 0.5, dict(kind=oracle.ISO_POINT, x0=(s[1] + 0.5) * dx, z0=(s[0] + 0.5) * dx),
                         RunParams(K=0, n_packets=300000, seed=7), with_variance=True)
    q = np.zeros((nz, nx), np.float32)
    q[d] = 1.0 / (2 * math.pi * dx * dx)
    adj = oracle.adjoint(mua, mus, dx, 0.5, q, RunParams(K=0, n_packets=300000, seed=8), with_variance=True)
    a, b = fwd.coeff[0][d], adj.coeff[0][s]
    assert abs(a - b) < 5 * math.sqrt(fwd.a0_var[d] + adj.a0_var[s]) + 0.01 * a


# ------------------------------------------------------- adjoint direction (Eq. 12)
def test_adjoint_radiance_points_back_to_source():
    """With mu_s = 0, Eq. 12 gives phi*(x, s) = int_0^inf q*(x + t s) e^{-mu_a t} dt: the adjoint
    radiance below a source pixel looks UP (theta = pi), so a*_1 ~ -a*_0 there, whereas the
    forward radiance of the same volumetric source points down (a_1 ~ +a_0)."""
    nz, nx, dx = 40, 9, 0.1
    mua, mus = np.full((nz, nx), 0.05), np.zeros((nz, nx))
    q = np.zeros((nz, nx), np.float32)
    q[1, 4] = 1.0
    run = RunParams(K=2, n_packets=200000, seed=4)
    adj = oracle.adjoint(mua, mus, dx, 0.0, q, run)
    fwd = oracle.volume(mua, mus, dx, 0.0, q, run, adjoint=False)
    for iz in (20, 30, 38):
        a0, a1, b1 = adj.coeff[0, iz, 4], adj.coeff[1, iz, 4], adj.coeff[2, iz, 4]
        assert a0 > 0 and a1 / a0 < -0.99 and abs(b1 / a0) < 0.05
        f0, f1 = fwd.coeff[0, iz, 4], fwd.coeff[1, iz, 4]
        assert f1 / f0 > 0.99
        assert abs(a0 - f0) < 1e-12 * f0  # a_0 does not depend on the direction convention
    # a_2 is even under theta -> theta + pi
    assert np.allclose(adj.coeff[3], fwd.coeff[3], rtol=1e-12, atol=1e-15)
    assert np.allclose(adj.coeff[1], -fwd.coeff[1], rtol=1e-12, atol=1e-15)


# -------------------------------------------------------- volumetric source sampling
def test_volume_sampler_follows_abs_q():
    """Adjoint launch pixels are drawn with probability |q*_i| / sum |q*| (Sec. 6, reading A5)."""
    rng = np.random.default_rng(0)
    q = (rng.normal(size=(3, 4)) * np.array([1, 0, 2, 0.5])).astype(np.float32)
    q[1, 1] = 0.0
    n = 20000
    picks = np.array([oracle.volume_pick(q, 5, 0, p) for p in range(n)])
    assert np.all(np.abs(q.ravel()[picks]) > 0)
    counts = np.bincount(picks, minlength=q.size).astype(float)
    p = np.abs(q.ravel()).astype(np.float64)
    p /= p.sum()
    nz = p > 0
    chi2 = np.sum((counts[nz] - n * p[nz]) ** 2 / (n * p[nz]))
    assert stats.chi2.sf(chi2, nz.sum() - 1) > 1e-4


# ------------------------------------------------------------ angular point sources (Sec. 4.1)
ANG_DENSITIES = [
    ([0.0, 0.0, 0.0, -1.0], []),      # sin^2(2 theta) / pi, the detector of Sec. 4.1
    ([], [1.0]),                      # (1 + sin theta) / (2 pi): odd under theta -> theta + pi
    ([0.3, 0.0, 0.2], [0.0, -0.4]),   # a mixture of cos and sin terms
]


def _ang(v, n):
    return v[n - 1] if n <= len(v) else 0.0


@pytest.mark.parametrize("ac,as_", ANG_DENSITIES)
def test_angular_point_source_launch_moments(ac, as_):
    """Launch directions follow p(theta) = (1 + sum_n c_n cos n theta + s_n sin n theta) / (2 pi):
    with absorption so strong that every packet leaves all its weight in the source pixel, that
    pixel's a_n / a_0 and b_n / a_0 are the sample means of cos n theta and sin n theta, whose
    expectations are c_n / 2 and s_n / 2."""
    n, dx, K, N = 5, 1.0, 6, 200000
    mua, mus = np.full((n, n), 1000.0), np.zeros((n, n))
    src = dict(kind=oracle.ANGULAR_POINT, x0=2.5, z0=2.5, ang_c=ac, ang_s=as_)
    r = oracle.forward(mua, mus, dx, 0.0, src, RunParams(K=K, n_packets=N, seed=21))
    a0 = r.coeff[0][2, 2]
    sig = 0.75 / math.sqrt(N)
    for m in range(1, K + 1):
        assert abs(r.coeff[2 * m - 1][2, 2] / a0 - _ang(ac, m) / 2) < 5 * sig, (m, r.coeff[2 * m - 1][2, 2] / a0)
        assert abs(r.coeff[2 * m][2, 2] / a0 - _ang(as_, m) / 2) < 5 * sig, (m, r.coeff[2 * m][2, 2] / a0)


def test_reciprocity_case2_angular_detectors():
    """Case 2 (Eqs. 15, 18): a unit isotropic point source at r_s and a unit point detector at r_d
    with angular sensitivity p(theta).  The detected signal  int phi(r_d, s) p(s) ds  is
    (a_0 + sum_n c_n a_n + s_n b_n)(r_d) / (2 pi); by reciprocity it equals Phi*(r_s) / (2 pi), and
    with the adjoint radiance read as phi*(r, s) = psi(r, -s) (reading A3) Phi*(r_s) is the fluence
    at r_s of a forward run from r_d with density p(theta + pi), coefficients (-1)^n c_n, (-1)^n s_n.
    The detector of Sec. 4.1 is even and cannot tell the flip; (1 + sin theta) / (2 pi) is odd and
    the identity fails without it."""
    nz = nx = 24
    dx, g, K = 0.25, 0.5, 4
    mua, mus = _hetero(nz, nx, 17)
    mua, mus = mua * 0.2, mus * 0.5
    ps, pd = (12, 12), (12, 18)  # (iz, ix): the detector 1.5 mm from the source along +x

    def centre(p):
        return dict(x0=(p[1] + 0.5) * dx, z0=(p[0] + 0.5) * dx)

    def flipped(v):
        return [(-1) ** n * x for n, x in enumerate(v, start=1)]

    for ac, as_ in ANG_DENSITIES[:2]:
        det, rec, unflipped = [], [], []
        for k in range(6):
            f = oracle.forward(mua, mus, dx, g, dict(kind=oracle.ISO_POINT, **centre(ps)),
                               RunParams(K=K, n_packets=60000, seed=50 + k))
            det.append(f.coeff[0][pd] + sum(_ang(ac, n) * f.coeff[2 * n - 1][pd] + _ang(as_, n) * f.coeff[2 * n][pd]
                                            for n in range(1, K + 1)))
            run = RunParams(K=0, n_packets=60000, seed=70 + k)
            rec.append(oracle.forward(mua, mus, dx, g, dict(kind=oracle.ANGULAR_POINT, **centre(pd), ang_c=flipped(ac),
                                                            ang_s=flipped(as_)), run).coeff[0][ps])
            unflipped.append(oracle.forward(mua, mus, dx, g, dict(kind=oracle.ANGULAR_POINT, **centre(pd), ang_c=ac,
                                                                  ang_s=as_), run).coeff[0][ps])
        det, rec, unflipped = map(np.array, (det, rec, unflipped))
        se = math.sqrt(det.var(ddof=1) / 6 + rec.var(ddof=1) / 6)
        assert abs(det.mean() - rec.mean()) < 4 * se + 0.01 * det.mean(), (ac, as_, det.mean(), rec.mean(), se)
        if as_:  # the odd detector: the missing flip is detected
            assert abs(det.mean() - unflipped.mean()) > 6 * se + 0.05 * det.mean(), (det.mean(), unflipped.mean(), se)


def _blob(nz, nx, dx, centre, sigma_px):
    """Unit-power distributed source density P_s [nz, nx] (sum P_s dx^2 = 1): a Gaussian blob."""
    iz, ix = np.mgrid[0:nz, 0:nx]
    p = np.exp(-((iz - centre[0]) ** 2 + (ix - centre[1]) ** 2) / (2.0 * sigma_px ** 2))
    return p / (p.sum() * dx * dx)


def test_reciprocity_case3_distributed_source_angular_detector():
    """Case 3 (Eqs. 16, 19): a distributed isotropic source a3 = P_s(r) / (2 pi) (unit power: the
    volumetric source q = P_s / (2 pi) per unit area and angle) and a point detector at r_d with
    angular sensitivity p(theta).  <L a3, b3> = (a_0 + sum_n c_n a_n + s_n b_n)(r_d) / (2 pi) of the
    forward run from the distributed source; <a3, L* b3> = sum_i dx^2 q_i Phi*_i, with Phi* the
    adjoint fluence of the detector -- the fluence of a forward run from r_d with density
    p(theta + pi) (reading A3).  So (a_0 + sum c_n a_n + s_n b_n)(r_d) = sum_i dx^2 P_s,i Phi*_i.
    (The printed Eq. 19 exchanges the roles of P_s and P_d; this is what Eq. 13 gives for the a3,
    b3 of Eq. 16.)  With the odd detector (1 + sin theta) / (2 pi) the identity fails without the
    turn by pi."""
    nz = nx = 24
    dx, g, K = 0.25, 0.5, 4
    mua, mus = _hetero(nz, nx, 19)
    mua, mus = mua * 0.2, mus * 0.5
    pd = (12, 18)
    Ps = _blob(nz, nx, dx, (12, 8), 1.5)
    q = (Ps / (2 * math.pi)).astype(np.float32)

    def flipped(v):
        return [(-1) ** n * x for n, x in enumerate(v, start=1)]

    centre = dict(x0=(pd[1] + 0.5) * dx, z0=(pd[0] + 0.5) * dx)
    for ac, as_ in ANG_DENSITIES[:2]:
        det, rec, unflipped = [], [], []
        for k in range(6):
            f = oracle.volume(mua, mus, dx, g, q, RunParams(K=K, n_packets=60000, seed=150 + k), adjoint=False)
            assert abs(f.source_strength - 1.0) < 1e-6
            det.append(f.coeff[0][pd] + sum(_ang(ac, n) * f.coeff[2 * n - 1][pd] + _ang(as_, n) * f.coeff[2 * n][pd]
                                            for n in range(1, K + 1)))
            run = RunParams(K=0, n_packets=60000, seed=170 + k)
            phi = oracle.forward(mua, mus, dx, g, dict(kind=oracle.ANGULAR_POINT, **centre, ang_c=flipped(ac),
                                                       ang_s=flipped(as_)), run).coeff[0]
            rec.append(float((Ps * phi).sum() * dx * dx))
            phi_u = oracle.forward(mua, mus, dx, g, dict(kind=oracle.ANGULAR_POINT, **centre, ang_c=ac, ang_s=as_),
                                   run).coeff[0]
            unflipped.append(float((Ps * phi_u).sum() * dx * dx))
        det, rec, unflipped = map(np.array, (det, rec, unflipped))
        se = math.sqrt(det.var(ddof=1) / 6 + rec.var(ddof=1) / 6)
        assert abs(det.mean() - rec.mean()) < 4 * se + 0.01 * det.mean(), (ac, as_, det.mean(), rec.mean(), se)
        if as_:  # the odd detector: the missing turn is detected
            assert abs(det.mean() - unflipped.mean()) > 6 * se + 0.05 * det.mean(), (det.mean(), unflipped.mean(), se)


# ------------------------------------------------------------ time-resolved fluence (Sec. 4.1 detectors)
def test_time_bins_partition_the_fluence():
    """The time-resolved tally splits each segment's track weight over path-length bins (the last
    open-ended): on the same packets the bins sum to a_0 (FP64 rounding), for bins much shorter
    and much longer than a pixel."""
    mua, mus, dx, g, src = _sector_case()
    h = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=5000, seed=5))
    for T, w in ((1, 0.5), (40, 0.01), (16, 0.7)):
        r = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=5000, seed=5, time_bins=T, time_bin_mm=w))
        assert r.coeff.shape[0] == T
        assert np.allclose(r.coeff.sum(axis=0), h.coeff[0], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("direction", ["down", "right"])
def test_time_bins_ballistic_closed_form(direction):
    """mu_s = 0: a collimated beam along an axis crosses pixel k over the path lengths
    [k dx, (k+1) dx); the fluence of that pixel in the bin [b w, (b+1) w) is the integral of
    e^{-mu_a L} over the overlap, divided by the pixel area (exact, every packet alike)."""
    n, dx, mu, T, w = 12, 0.1, 0.7, 7, 0.13
    mua, mus = np.full((n, n), mu), np.zeros((n, n))
    if direction == "down":
        src = dict(kind=oracle.PENCIL, x0=0.45, z0=0.0, dir_x=0.0, dir_z=1.0)
    else:
        src = dict(kind=oracle.PENCIL, x0=0.0, z0=0.75, dir_x=1.0, dir_z=0.0)
    r = oracle.forward(mua, mus, dx, 0.3, src, RunParams(K=0, n_packets=16, seed=1, time_bins=T, time_bin_mm=w))
    line = r.coeff[:, :, 4] if direction == "down" else r.coeff[:, 7, :]
    want = np.zeros((T, n))
    for k in range(n):
        for b in range(T):
            lo, hi = max(k * dx, b * w), min((k + 1) * dx, (b + 1) * w if b < T - 1 else np.inf)
            if hi > lo:
                want[b, k] = (math.exp(-mu * lo) - math.exp(-mu * hi)) / mu / (dx * dx)
    assert np.allclose(line, want, rtol=1e-12, atol=1e-14)
    off = r.coeff.copy()
    if direction == "down":
        off[:, :, 4] = 0
    else:
        off[:, 7, :] = 0
    assert not off.any()


def test_time_bins_decay_with_absorption():
    """Paths do not depend on mu_a (absorption weighting, reading 1), so with roulette off and the
    same packets, a pixel's fluence in path-length bin b with uniform mu_a is the mu_a = 0 one
    weighted by e^{-mu_a L} over that bin: their ratio lies in [e^{-mu_a (b+1) w}, e^{-mu_a b w}]."""
    n, dx, g, T, w, mu = 16, 0.1, 0.6, 12, 0.35, 0.8
    mus = _hetero(n, n, 29)[1]
    src = dict(kind=oracle.ISO_POINT, x0=0.83, z0=0.77)
    run = RunParams(K=0, n_packets=4000, seed=12, w_threshold=0.0, time_bins=T, time_bin_mm=w)
    f0 = oracle.forward(np.zeros((n, n)), mus, dx, g, src, run).coeff
    fa = oracle.forward(np.full((n, n), mu), mus, dx, g, src, run).coeff
    for b in range(T - 1):
        m = f0[b] > 0
        ratio = fa[b][m] / f0[b][m]
        assert ratio.min() >= math.exp(-mu * (b + 1) * w) * (1 - 1e-12), b
        assert ratio.max() <= math.exp(-mu * b * w) * (1 + 1e-12), b
    assert (fa[T - 1] <= f0[T - 1] * math.exp(-mu * (T - 1) * w) * (1 + 1e-12)).all()
    assert ((f0 > 0) == (fa > 0)).all()


# ------------------------------------------------------------ discrete ordinates (Sec. 3.1)
def _sector_case():
    nz = nx = 20
    dx, g = 0.2, 0.7
    mua, mus = _hetero(nz, nx, 23)
    src = dict(kind=oracle.ISO_POINT, x0=2.1, z0=1.9)
    return mua * 0.3, mus, dx, g, src


def test_sectors_partition_the_fluence_deposits():
    """The discrete-ordinates tally (the alternative Sec. 3.1 sets aside) splits every deposit of
    Eq. 9 into exactly one sector: on the same packets the sectors sum to a_0 (FP64 rounding)."""
    mua, mus, dx, g, src = _sector_case()
    h = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=20000, seed=5))
    for M in (1, 6, 32):
        s = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=20000, seed=5, sectors=M))
        assert s.coeff.shape[0] == M
        assert np.allclose(s.coeff.sum(axis=0), h.coeff[0], rtol=1e-12, atol=1e-15)


def test_sectors_equal_the_harmonic_series_integrated_over_each_sector():
    """On the same packets the sector integrals of the radiance equal the integrals over each
    sector of its Fourier series (Eq. 8) with coefficients of Eqs. 9-11 up to K = 64; what is
    left is the series' truncation near the sector edges, small where the field is diffuse."""
    mua, mus, dx, g, src = _sector_case()
    K, M, N = 64, 8, 40000
    h = oracle.forward(mua, mus, dx, g, src, RunParams(K=K, n_packets=N, seed=8))
    s = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=N, seed=8, sectors=M))
    dth = 2 * math.pi / M
    region = (slice(12, 20), slice(12, 20))  # away from the source: a diffuse field
    for m in range(M):
        t1, t2 = m * dth, (m + 1) * dth
        series = h.coeff[0] * dth / (2 * math.pi)
        for n in range(1, K + 1):
            series = series + (h.coeff[2 * n - 1] * (math.sin(n * t2) - math.sin(n * t1))
                               - h.coeff[2 * n] * (math.cos(n * t2) - math.cos(n * t1))) / (n * math.pi)
        a, b = s.coeff[m][region].sum(), series[region].sum()
        assert abs(a - b) < 0.01 * abs(a), (m, a, b)


def test_sector_estimates_converge_slower_than_the_fluence():
    """Sec. 3.1: the per-sector radiance estimate has a larger relative spread than the fluence
    estimate from the same packets, and the gap grows with the number of sectors."""
    mua, mus, dx, g, src = _sector_case()
    pix = (14, 15)

    def rel_sd(M):
        vals = []
        for k in range(8):
            r = oracle.forward(mua, mus, dx, g, src, RunParams(K=0, n_packets=4000, seed=300 + k, sectors=M))
            vals.append(r.coeff[0][pix] if M == 0 else r.coeff[:, pix[0], pix[1]])
        v = np.array(vals)
        return float(np.mean(v.std(axis=0, ddof=1) / np.abs(v.mean(axis=0))))

    r0, r4, r16 = rel_sd(0), rel_sd(4), rel_sd(16)
    assert r0 < r4 < r16, (r0, r4, r16)
