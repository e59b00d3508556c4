"""Pixelwise functionals of the oracle, in FP64 numpy (TEST INFRASTRUCTURE ONLY).

Each function is the paper's formula written out, with no blocking or fusion:

* ``absorbed_energy``  H = mu_a Phi, Phi = a_0                         (Sec. 2, Sec. 5)
* ``error_functional`` eps = 1/2 int (H^meas - H)^2 dx, pixel sums     (Eq. 2)
* ``grad_mua_paper``   d eps / d mu_a, per unit area                  (Eq. 22)
* ``grad_mus_paper``   d eps / d mu_s, per unit area                  (Eq. 28)
* ``adjoint_source_paper``  q* = mu_a (H^meas - H)                      (Sec. 6)
* ``G_a``, ``G_s``     the angular integrals int phi* phi ds and
                        int phi* phi ds - int int phi* P phi ds' ds   (Eqs. 22, 26, 28)
* ``dL_dmu``           gradients of a general pixel loss L(H) with v = dL/dH_i:
                        q*_i = -mu_a,i v_i / A,  dL/dmu_a,i = v_i a_0,i + A G_a,i,
                        dL/dmu_s,i = A G_s,i.  For L = eps (v_i = -A (H^meas_i - H_i)) this
                        is A times Eqs. 22 and 28 (derivation: Sec. 2 gradients, Eqs. 3-4,
                        with the adjoint of Eq. 12 driven by the pixel-constant source).

Coefficient arrays are [2K+1, nz, nx] with channel 0 = a_0, 2n-1 = a_n, 2n = b_n; the truncation
of the infinite sums at n = K is the reading taken for the paper's infinite series.
Sums over n run in increasing n.
"""
from __future__ import annotations

import math

import numpy as np


def _split(coeff):
    coeff = np.asarray(coeff, dtype=np.float64)
    K = (coeff.shape[0] - 1) // 2
    a0 = coeff[0]
    a = [coeff[2 * n - 1] for n in range(1, K + 1)]
    b = [coeff[2 * n] for n in range(1, K + 1)]
    return K, a0, a, b


def absorbed_energy(mua, coeff):
    """H = mu_a a_0 (Sec. 2 with Grueneisen parameter 1; a_0 is the fluence, Sec. 5)."""
    return np.asarray(mua, dtype=np.float64) * np.asarray(coeff, dtype=np.float64)[0]


def error_functional(Hmeas, H, dx):
    """eps = 1/2 sum_i A (H^meas_i - H_i)^2, the pixel form of Eq. 2."""
    r = np.asarray(Hmeas, dtype=np.float64) - np.asarray(H, dtype=np.float64)
    return 0.5 * dx * dx * float(np.sum(r * r))


def G_a(coeff, coeff_adj):
    """int phi phi* ds = a_0 a_0*/(2 pi) + (1/pi) sum_n (a_n a_n* + b_n b_n*)  (Eq. 22)."""
    K, a0, a, b = _split(coeff)
    K2, s0, sa, sb = _split(coeff_adj)
    assert K == K2
    out = a0 * s0 / (2.0 * math.pi)
    for n in range(K):
        out = out + (a[n] * sa[n] + b[n] * sb[n]) / math.pi
    return out


def G_s(coeff, coeff_adj, g):
    """int phi* phi ds - int int phi* P phi = (1/pi) sum_n (a_n a_n* + b_n b_n*)(1 - g^n)  (Eq. 28)."""
    K, a0, a, b = _split(coeff)
    K2, s0, sa, sb = _split(coeff_adj)
    assert K == K2
    out = np.zeros_like(a0)
    for n in range(1, K + 1):
        out = out + (a[n - 1] * sa[n - 1] + b[n - 1] * sb[n - 1]) * (1.0 - g ** n) / math.pi
    return out


def scatter_term(coeff, coeff_adj, g):
    """int int phi*(s) P(s, s') phi(s') ds' ds = a_0 a_0*/(2 pi) + (1/pi) sum_n g^n (...)  (Eq. 26)."""
    K, a0, a, b = _split(coeff)
    _, s0, sa, sb = _split(coeff_adj)
    out = a0 * s0 / (2.0 * math.pi)
    for n in range(1, K + 1):
        out = out + (a[n - 1] * sa[n - 1] + b[n - 1] * sb[n - 1]) * g ** n / math.pi
    return out


def grad_mua_paper(coeff, coeff_adj, mua, Hmeas):
    """d eps / d mu_a = -a_0 (H^meas - mu_a a_0) + a_0 a_0*/(2 pi) + (1/pi) sum (a_n a_n* + b_n b_n*)  (Eq. 22)."""
    a0 = np.asarray(coeff, dtype=np.float64)[0]
    mua = np.asarray(mua, dtype=np.float64)
    return -a0 * (np.asarray(Hmeas, dtype=np.float64) - mua * a0) + G_a(coeff, coeff_adj)


def grad_mus_paper(coeff, coeff_adj, g):
    """d eps / d mu_s = (1/pi) sum_n (a_n a_n* + b_n b_n*)(1 - g^n)  (Eq. 28)."""
    return G_s(coeff, coeff_adj, g)


def adjoint_source_paper(mua, Hmeas, H):
    """q* = mu_a (H^meas - H), isotropic, per unit area and unit angle (Sec. 6)."""
    return np.asarray(mua, dtype=np.float64) * (np.asarray(Hmeas, dtype=np.float64) - np.asarray(H, dtype=np.float64))


def dL_dH_eps(Hmeas, H, dx):
    """v_i = d eps / d H_i for the pixel form of Eq. 2: v_i = -A (H^meas_i - H_i)."""
    return -dx * dx * (np.asarray(Hmeas, dtype=np.float64) - np.asarray(H, dtype=np.float64))


def adjoint_source(mua, v, dx):
    """q*_i = -mu_a,i v_i / A for a pixel loss with v = dL/dH (equals Sec. 6's q* when L = eps)."""
    return -np.asarray(mua, dtype=np.float64) * np.asarray(v, dtype=np.float64) / (dx * dx)


def dL_dmu(coeff, coeff_adj, v, dx, g):
    """(dL/dmu_a, dL/dmu_s) per pixel for a pixel loss with v = dL/dH (discrete, x pixel area)."""
    A = dx * dx
    a0 = np.asarray(coeff, dtype=np.float64)[0]
    d_mua = np.asarray(v, dtype=np.float64) * a0 + A * G_a(coeff, coeff_adj)
    d_mus = A * G_s(coeff, coeff_adj, g)
    return d_mua, d_mus


# ---------------------------------------------------------------------------------------------- 3D
# The 3D form (the extension Sec. 3.1 names): coefficients [(L+1)^2, nz, ny, nx] of orthonormal
# real spherical harmonics, phi(s) = sum c_lm Y_lm(s); fluence sqrt(4 pi) c_00; the HG kernel is
# sum_l g^l sum_m Y_lm(s) Y_lm(s'), so the angular integrals of Eqs. 22, 26, 28 become sums of
# c_lm c*_lm (weighted by g^l for the scattering term).  Voxel volume V = dx^3.
def _l_of(C):
    return np.array([int(math.isqrt(c)) for c in range(C)])


def fluence3(coeff):
    """Phi = int phi ds = sqrt(4 pi) c_00."""
    return math.sqrt(4.0 * math.pi) * np.asarray(coeff, dtype=np.float64)[0]


def absorbed_energy3(mua, coeff):
    """H = mu_a Phi (Sec. 2) in 3D."""
    return np.asarray(mua, dtype=np.float64) * fluence3(coeff)


def error_functional3(Hmeas, H, dx):
    """eps = 1/2 sum_v V (H^meas_v - H_v)^2 (Eq. 2 over voxels)."""
    r = np.asarray(Hmeas, dtype=np.float64) - np.asarray(H, dtype=np.float64)
    return 0.5 * dx ** 3 * float(np.sum(r * r))


def dL_dH_eps3(Hmeas, H, dx):
    """dL/dH_v for L = eps: -V (H^meas_v - H_v)."""
    return -dx ** 3 * (np.asarray(Hmeas, dtype=np.float64) - np.asarray(H, dtype=np.float64))


def adjoint_source3(mua, v, dx):
    """q*_v = -mu_a,v v_v / V, per unit volume and solid angle (isotropic)."""
    return -np.asarray(mua, dtype=np.float64) * np.asarray(v, dtype=np.float64) / dx ** 3


def G_a3(coeff, coeff_adj):
    """int phi phi* ds = sum_lm c_lm c*_lm (orthonormal basis), in increasing channel order."""
    c, a = np.asarray(coeff, dtype=np.float64), np.asarray(coeff_adj, dtype=np.float64)
    out = np.zeros(c.shape[1:])
    for k in range(c.shape[0]):
        out = out + c[k] * a[k]
    return out


def G_s3(coeff, coeff_adj, g):
    """int phi* phi ds - int int phi* P phi = sum_lm (1 - g^l) c_lm c*_lm."""
    c, a = np.asarray(coeff, dtype=np.float64), np.asarray(coeff_adj, dtype=np.float64)
    ls = _l_of(c.shape[0])
    out = np.zeros(c.shape[1:])
    for k in range(c.shape[0]):
        out = out + (1.0 - g ** int(ls[k])) * c[k] * a[k]
    return out


def dL_dmu3(coeff, coeff_adj, v, dx, g):
    """Gradients of a voxel loss L(H) with v = dL/dH: dL/dmu_a = v Phi + V G_a, dL/dmu_s = V G_s."""
    V = dx ** 3
    ga = np.asarray(v, dtype=np.float64) * fluence3(coeff) + V * G_a3(coeff, coeff_adj)
    gs = V * G_s3(coeff, coeff_adj, g)
    return ga, gs
