"""Seeded synthetic inputs shaped like the paper's phantoms (no dataset exists for this method).

This module holds input generators only -- pixel maps, source descriptors and run sizes -- and
none of the method's arithmetic; the CUDA path and the oracle both draw their inputs from it.
The paper's phantoms (Sec. 6.1, 6.2: background mu_a 0.01/mm, inclusions of 0.2/mm, mu_s 5 -> 15
/mm, g = 0.9, collimated line sources) are under-specified, so the media below are synthetic
stand-ins of the same kind: a homogeneous background with random circular inclusions, or a
smooth lognormal random field.

Workloads (sizes in pixels, dx in mm):
  * ``pencil32``  32x32 of 0.25 mm, mu_a 0.01, mu_s 5, g 0.8, pencil beam at the top centre,
                  K = 8, 1e5 packets, seed 0.
  * ``grad256``   256x256 of 0.05 mm (12.8 mm), background mu_a 0.01 / mu_s 10, g 0.9,
                  3 random circular inclusions (mu_a 0.02-0.2, mu_s 5-20), collimated line source
                  on the top edge, K = 32, 1e7 packets forward + 1e7 adjoint, gradient.
  * ``large1024`` 1024x1024 of 0.02 mm, same background, 8 inclusions (mu_s <= 20), K = 64,
                  1e9 packets, four line sources (one per edge).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PENCIL, LINE, ISO_POINT, ANGULAR_POINT = 0, 1, 2, 3


@dataclass
class Workload:
    name: str
    nx: int
    nz: int
    dx: float
    g: float
    K: int
    n_packets: int
    mua: np.ndarray          # current estimate [nz, nx] float32
    mus: np.ndarray
    sources: list            # list of source dicts (kind, x0, z0, x1, z1, dir_x, dir_z, power)
    mua_true: np.ndarray | None = None   # phantom that generates H^meas (gradient workloads)
    mus_true: np.ndarray | None = None
    seed: int = 0
    meta: dict = field(default_factory=dict)


def inclusion_phantom(n: int, dx: float, n_incl: int, seed: int, mua_bg=0.01, mus_bg=10.0,
                      mua_range=(0.02, 0.2), mus_range=(5.0, 20.0), radius=(0.5, 1.5), margin=2.0):
    """Homogeneous background with circular inclusions (later ones overwrite earlier ones).

    Centres uniform in [margin, L - margin]^2 (L = n dx), radii uniform in ``radius`` (mm),
    inclusion mu_a / mu_s uniform in the given ranges; numpy ``default_rng(seed)``.
    """
    rng = np.random.default_rng(seed)
    L = n * dx
    c = (np.arange(n) + 0.5) * dx
    X, Z = np.meshgrid(c, c)
    mua = np.full((n, n), mua_bg, np.float64)
    mus = np.full((n, n), mus_bg, np.float64)
    for _ in range(n_incl):
        cx, cz = rng.uniform(margin, L - margin, 2)
        r = rng.uniform(*radius)
        a = rng.uniform(*mua_range)
        s = rng.uniform(*mus_range)
        m = (X - cx) ** 2 + (Z - cz) ** 2 <= r * r
        mua[m] = a
        mus[m] = s
    return mua.astype(np.float32), mus.astype(np.float32)


def lognormal_field(n: int, dx: float, mean: float, sigma: float, corr_mm: float, seed: int):
    """mean * exp(sigma G - sigma^2/2), G a unit-variance Gaussian random field with squared-
    exponential correlation of length corr_mm, made by FFT-filtering seeded white noise."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, d=dx) * 2 * np.pi
    KX, KZ = np.meshgrid(k, k)
    filt = np.exp(-(KX ** 2 + KZ ** 2) * corr_mm ** 2 / 4.0)
    G = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    G = (G - G.mean()) / (G.std() + 1e-30)
    return (mean * np.exp(sigma * G - 0.5 * sigma * sigma)).astype(np.float32)


def residual_source(n: int, dx: float, seed: int, mua_bg: float = 0.01, depth_mm: float = 3.0):
    """Signed isotropic source [n, n] (float32, per unit area and angle) shaped like the adjoint
    source q* = mu_a (H^meas - H) of a reconstruction (Sec. 6): a mixture, with random weights, of
    (a) the mu_a contrast of 1-4 random circular inclusions times an exponential decay with depth
    (the fluence under a top line source), (b) a smooth zero-mean Gaussian random field (1 mm
    correlation) with the same decay, and (c) pixel-scale white noise (the residual left once the
    noise of H^meas and H dominates), with a random overall sign; ``default_rng(seed)``.
    Scale: |q| ~ mu_a_bg^2 exp(-z / depth_mm).  Input generator only (no transport)."""
    rng = np.random.default_rng(seed)
    c = (np.arange(n) + 0.5) * dx
    decay = np.exp(-c / depth_mm)[:, None] * np.ones((1, n))
    mua, _ = inclusion_phantom(n, dx, int(rng.integers(1, 5)), seed=int(rng.integers(1 << 30)),
                               mua_bg=mua_bg, mua_range=(0.005, 0.2), margin=min(2.0, 0.15 * n * dx))
    contrast = (mua.astype(np.float64) - mua_bg) / mua_bg
    field = lognormal_field(n, dx, 1.0, 1.0, 1.0, seed=int(rng.integers(1 << 30))).astype(np.float64)
    smooth = np.log(np.maximum(field, 1e-30))
    smooth = (smooth - smooth.mean()) / (smooth.std() + 1e-30)
    white = rng.standard_normal((n, n))
    w = rng.dirichlet((1.0, 1.0, 1.0))
    q = (w[0] * contrast + w[1] * 0.5 * smooth + w[2] * 0.5 * white) * decay * mua_bg * mua_bg
    return (q * (1.0 if rng.uniform() < 0.5 else -1.0)).astype(np.float32)


def top_line_source(nx: int, dx: float) -> dict:
    return dict(kind=LINE, x0=0.0, z0=0.0, x1=nx * dx, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)


def edge_line_sources(n: int, dx: float, per_edge: int = 1) -> list:
    """``per_edge`` equal collimated line sources on each of the four edges, pointing inward."""
    L = n * dx
    out = []
    for k in range(per_edge):
        a, b = k * L / per_edge, (k + 1) * L / per_edge
        out.append(dict(kind=LINE, x0=a, z0=0.0, x1=b, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0))   # top, +z
        out.append(dict(kind=LINE, x0=a, z0=L, x1=b, z1=L, dir_x=0.0, dir_z=-1.0, power=1.0))     # bottom, -z
        out.append(dict(kind=LINE, x0=0.0, z0=a, x1=0.0, z1=b, dir_x=1.0, dir_z=0.0, power=1.0))   # left, +x
        out.append(dict(kind=LINE, x0=L, z0=a, x1=L, z1=b, dir_x=-1.0, dir_z=0.0, power=1.0))     # right, -x
    return out


def rect_phantom(n: int = 80, dx: float = 0.05):
    """The test domain of the reconstructions of Sec. 6: 4 mm x 4 mm (n = 80 pixels of 0.05 mm),
    background mu_a 0.01 and mu_s 5 /mm with a rectangular mu_a inclusion of 0.2 /mm and a
    rectangular mu_s inclusion of 15 /mm, g 0.9, lit by two equal collimated line sources on
    adjacent edges: z = 0 (pointing +z) and x = 4 mm (pointing -x).  The inclusions' positions
    are not given in the text (the figures are not available): the mu_a rectangle spans
    x in [1, 2] mm, z in [1, 2] mm (the paper's mu_a profile is taken at x = 1.5 mm), the mu_s
    rectangle x in [2, 3] mm, z in [1.5, 2.5] mm (its profile at x = 2.5 mm).
    Returns (mua, mus, g, sources)."""
    L = n * dx
    c = (np.arange(n) + 0.5) * dx
    X, Z = np.meshgrid(c, c)  # [iz][ix]
    mua = np.full((n, n), 0.01, np.float32)
    mus = np.full((n, n), 5.0, np.float32)
    mua[(X >= 1.0) & (X <= 2.0) & (Z >= 1.0) & (Z <= 2.0)] = 0.2
    mus[(X >= 2.0) & (X <= 3.0) & (Z >= 1.5) & (Z <= 2.5)] = 15.0
    srcs = [dict(kind=LINE, x0=0.0, z0=0.0, x1=L, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0),
            dict(kind=LINE, x0=L, z0=0.0, x1=L, z1=L, dir_x=-1.0, dir_z=0.0, power=1.0)]
    return mua, mus, 0.9, srcs


def pencil32() -> Workload:
    n, dx = 32, 0.25
    mua = np.full((n, n), 0.01, np.float32)
    mus = np.full((n, n), 5.0, np.float32)
    src = dict(kind=PENCIL, x0=n * dx / 2, z0=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    return Workload("pencil32", n, n, dx, 0.8, 8, 100_000, mua, mus, [src], seed=0)


def grad256(n_packets: int = 10_000_000) -> Workload:
    n, dx = 256, 0.05
    mua_t, mus_t = inclusion_phantom(n, dx, 3, seed=1)
    mua = np.full((n, n), 0.01, np.float32)   # starting estimate: the background
    mus = np.full((n, n), 10.0, np.float32)
    return Workload("grad256", n, n, dx, 0.9, 32, n_packets, mua, mus, [top_line_source(n, dx)],
                    mua_true=mua_t, mus_true=mus_t, seed=0, meta=dict(hmeas_seed=1001))


def large1024(n_packets: int = 1_000_000_000) -> Workload:
    n, dx = 1024, 0.02
    mua_t, mus_t = inclusion_phantom(n, dx, 8, seed=5, radius=(0.5, 2.5))
    mua = np.full((n, n), 0.01, np.float32)
    mus = np.full((n, n), 10.0, np.float32)
    return Workload("large1024", n, n, dx, 0.9, 64, n_packets, mua, mus, edge_line_sources(n, dx),
                    mua_true=mua_t, mus_true=mus_t, seed=0, meta=dict(hmeas_seed=1001))


def batch64(n_packets: int = 1_000_000, extent_mm: float = 12.8):
    """64 forward problems: 16 collimated line sources (4 per edge, each a quarter of the edge,
    pointing inward) x 4 wavelengths, on grids of 128^2 / 256^2 / 512^2 pixels taken round-robin
    over the problems at a fixed extent.  mu_a and mu_s are lognormal Gaussian random fields
    (sigma 0.5, correlation 1 mm, seed = problem index) around 0.01 and 10 /mm, scaled per
    wavelength by (0.5, 1, 1.5, 2) and (1.2, 1.0, 0.9, 0.8); g = 0.9; K = 16.

    Returns a list of dicts: nx, dx, mua, mus, g, source, n_packets, seed, stream_id.
    """
    sizes = (128, 256, 512)
    a_scale = (0.5, 1.0, 1.5, 2.0)
    s_scale = (1.2, 1.0, 0.9, 0.8)
    out = []
    for i in range(64):
        n = sizes[i % 3]
        dx = extent_mm / n
        srcs = edge_line_sources(n, dx, per_edge=4)
        src = srcs[(i // 4) % 16]
        wl = i % 4
        mua = lognormal_field(n, dx, 0.01, 0.5, 1.0, seed=i) * a_scale[wl]
        mus = lognormal_field(n, dx, 10.0, 0.5, 1.0, seed=1000 + i) * s_scale[wl]
        out.append(dict(nx=n, dx=dx, mua=mua.astype(np.float32), mus=mus.astype(np.float32), g=0.9,
                        source=src, n_packets=n_packets, seed=0, stream_id=2 * i))
    return out


def small_hetero(nz: int, nx: int, dx: float, seed: int):
    """Heterogeneous test medium: smooth background plus two rectangles (parity tests)."""
    rng = np.random.default_rng(seed)
    c_x = (np.arange(nx) + 0.5) * dx
    c_z = (np.arange(nz) + 0.5) * dx
    X, Z = np.meshgrid(c_x, c_z)
    mua = 0.05 + 0.04 * np.sin(X * 2.1 + rng.uniform(0, 6)) * np.cos(Z * 1.3)
    mus = 6.0 + 3.0 * np.cos(X * 1.7 - Z * 0.9 + rng.uniform(0, 6))
    i0, j0 = nz // 4, nx // 5
    mua[i0:i0 + nz // 3, j0:j0 + nx // 4] = 0.3
    mus[nz // 2:nz // 2 + nz // 4, nx // 2:nx // 2 + nx // 3] = 15.0
    return mua.astype(np.float32), mus.astype(np.float32)


def small_hetero3(nz: int, ny: int, nx: int, dx: float, seed: int):
    """Heterogeneous voxel medium for the 3D parity tests: smooth background plus a strongly
    absorbing box and a strongly scattering box (float32 [nz, ny, nx])."""
    rng = np.random.default_rng(seed)
    cz, cy, cx = ((np.arange(n) + 0.5) * dx for n in (nz, ny, nx))
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    ph = rng.uniform(0, 6, 3)
    mua = 0.05 + 0.04 * np.sin(2.1 * X + ph[0]) * np.cos(1.3 * Z + ph[1]) * np.cos(1.1 * Y)
    mus = 6.0 + 3.0 * np.cos(1.7 * X - 0.9 * Z + 1.2 * Y + ph[2])
    mua[nz // 4:nz // 4 + max(1, nz // 3), ny // 3:ny // 3 + max(1, ny // 4), nx // 5:nx // 5 + max(1, nx // 4)] = 0.3
    mus[nz // 2:nz // 2 + max(1, nz // 4), :ny // 2, nx // 2:nx // 2 + max(1, nx // 3)] = 15.0
    return mua.astype(np.float32), mus.astype(np.float32)


def phantom3(n: int, dx: float, seed: int):
    """3D gradient workload on n^3 voxels of side dx: a scattering background (mu_s 10/mm,
    mu_a 0.01/mm with +-20% smooth variation) and, in the 'true' medium, three absorbing spheres
    (mu_a x 3); a pencil beam enters the top face at the centre of its middle voxel (not on a voxel
    face, where FP32 and FP64 would start it in different voxels).  Returns (mua, mus, mua_true,
    source dict), the maps float32 [nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    ext = n * dx
    ph = rng.uniform(0, 2 * np.pi, 3)
    k = 2 * np.pi / ext
    mua = 0.01 * (1 + 0.2 * np.sin(k * X + ph[0]) * np.cos(k * Y + ph[1]) * np.cos(k * Z + ph[2]))
    mus = np.full_like(mua, 10.0)
    mua_true = mua.copy()
    for _ in range(3):
        ctr = rng.uniform(0.25, 0.75, 3) * ext
        r = rng.uniform(0.06, 0.12) * ext
        inside = (Z - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 + (X - ctr[2]) ** 2 < r * r
        mua_true[inside] *= 3.0
    xc = float(np.float32((n // 2 + 0.5) * dx))
    src = dict(kind=0, x0=xc, y0=xc, z0=0.0, dir_x=0.0, dir_y=0.0, dir_z=1.0, power=1.0)
    return mua.astype(np.float32), mus.astype(np.float32), mua_true.astype(np.float32), src
