"""Thin Python binding of the 3D calls of libmcr (include/mcr3.h): argument marshalling only.

The 3D form of the method (Sec. 3.1 names it: the Fourier angular basis of 2D becomes real
spherical harmonics): voxel maps ``mua``/``mus`` [nz, ny, nx] (float32 CUDA, 1/mm), voxel side
``dx`` (mm), 3D Henyey-Greenstein ``g``; coefficient tensors [(L+1)^2, nz, ny, nx] at channel
l^2 + l + m.  ``Run.K`` carries the order L.  Every step runs in the CUDA library; a negative
status raises :class:`mcr.McrError`, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import mcr
from .mcr import ISO_POINT, PENCIL, McrError, Run  # noqa: F401  (re-exported)

MAX_L = 8

# every symbol declared in include/mcr3.h
EXPORTS = ("mc3_forward", "mc3_adjoint", "mc3_h_eps", "mc3_adjoint_source", "mc3_gradient", "mc3_gradient_f32")


class _Medium3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_float), ("g", C.c_float),
                ("mua", C.c_void_p), ("mus", C.c_void_p)]


class _Source3(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_float), ("y0", C.c_float), ("z0", C.c_float),
                ("dir_x", C.c_float), ("dir_y", C.c_float), ("dir_z", C.c_float), ("power", C.c_float)]


_typed = False


def load() -> C.CDLL:
    """libmcr with the 3D entry points typed; raises if the library is not built."""
    global _typed
    lib = mcr.load()
    if not _typed:
        vp = C.c_void_p
        lib.mc3_forward.argtypes = [C.POINTER(_Medium3), C.POINTER(_Source3), C.POINTER(mcr._Run), vp,
                                    C.POINTER(mcr._Stats), vp]
        lib.mc3_adjoint.argtypes = [C.POINTER(_Medium3), vp, C.POINTER(mcr._Run), vp, C.POINTER(mcr._Stats), vp]
        lib.mc3_h_eps.argtypes = [C.POINTER(_Medium3), vp, vp, vp, vp, vp, vp]
        lib.mc3_adjoint_source.argtypes = [C.POINTER(_Medium3), vp, vp, vp]
        lib.mc3_gradient.argtypes = [C.POINTER(_Medium3), C.c_int32, vp, vp, vp, vp, vp, vp]
        lib.mc3_gradient_f32.argtypes = [C.POINTER(_Medium3), C.c_int32, vp, vp, vp, vp, vp, vp]
        for name in EXPORTS:
            getattr(lib, name).restype = C.c_int
        _typed = True
    return lib


@dataclass
class Medium3:
    """Voxel medium: mu_a, mu_s [nz, ny, nx] (float32 CUDA), voxel side dx, 3D HG g."""
    mua: torch.Tensor
    mus: torch.Tensor
    dx: float
    g: float

    @property
    def shape(self):
        return tuple(self.mua.shape)

    def c(self) -> _Medium3:
        mcr._dev_f32(self.mua, "mua")
        mcr._dev_f32(self.mus, "mus")
        if self.mua.shape != self.mus.shape or self.mua.dim() != 3:
            raise ValueError("mua and mus must have the same [nz, ny, nx] shape")
        nz, ny, nx = self.mua.shape
        return _Medium3(nx, ny, nz, float(self.dx), float(self.g), self.mua.data_ptr(), self.mus.data_ptr())


@dataclass
class Source3:
    """PENCIL (collimated along dir, normalised by the library) or ISO_POINT at (x0, y0, z0) mm."""
    kind: int
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    dir_x: float = 0.0
    dir_y: float = 0.0
    dir_z: float = 1.0
    power: float = 1.0

    def c(self) -> _Source3:
        return _Source3(int(self.kind), self.x0, self.y0, self.z0, self.dir_x, self.dir_y, self.dir_z, self.power)


def _coeff_out(med: Medium3, L: int, out):
    shape = ((L + 1) ** 2,) + med.shape
    if out is None:
        return torch.empty(shape, dtype=torch.float32, device=med.mua.device)
    mcr._dev_f32(out, "out")
    if tuple(out.shape) != shape:
        raise ValueError("out must be [(L+1)^2, nz, ny, nx]")
    return out


def forward(med: Medium3, src: Source3, run: Run, out=None, stats: bool = False, stream=None):
    """3D forward radiance MC (``mc3_forward``): coeff [(L+1)^2, nz, ny, nx] (and stats dict), L = run.K."""
    lib = load()
    coeff = _coeff_out(med, run.K, out)
    st = mcr._Stats() if stats else None
    rc = lib.mc3_forward(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), mcr._ptr(coeff),
                         C.byref(st) if st is not None else None, mcr._stream(stream))
    mcr._check(rc, "mc3_forward")
    return (coeff, mcr._stats_dict(st)) if stats else coeff


def adjoint(med: Medium3, qstar: torch.Tensor, run: Run, out=None, stats: bool = False, stream=None):
    """3D adjoint radiance MC from q* (``mc3_adjoint``): coeff_adj, tallied at -s."""
    lib = load()
    mcr._dev_f32(qstar, "qstar")
    if tuple(qstar.shape) != med.shape:
        raise ValueError("qstar must have the medium's shape")
    coeff = _coeff_out(med, run.K, out)
    st = mcr._Stats() if stats else None
    rc = lib.mc3_adjoint(C.byref(med.c()), mcr._ptr(qstar), C.byref(run.c()), mcr._ptr(coeff),
                         C.byref(st) if st is not None else None, mcr._stream(stream))
    mcr._check(rc, "mc3_adjoint")
    return (coeff, mcr._stats_dict(st)) if stats else coeff


def h_eps(med: Medium3, coeff: torch.Tensor, Hmeas: torch.Tensor | None = None, stream=None):
    """H = mu_a sqrt(4 pi) c_00; with Hmeas also dL/dH = -dx^3 (Hmeas - H) and eps (``mc3_h_eps``)."""
    lib = load()
    mcr._dev_f32(coeff, "coeff")
    H = torch.empty(med.shape, dtype=torch.float32, device=coeff.device)
    if Hmeas is None:
        mcr._check(lib.mc3_h_eps(C.byref(med.c()), mcr._ptr(coeff), None, mcr._ptr(H), None, None,
                                 mcr._stream(stream)), "mc3_h_eps")
        return H
    mcr._dev_f32(Hmeas, "Hmeas")
    v = torch.empty_like(H)
    eps = torch.empty((), dtype=torch.float64, device=coeff.device)
    mcr._check(lib.mc3_h_eps(C.byref(med.c()), mcr._ptr(coeff), mcr._ptr(Hmeas), mcr._ptr(H), mcr._ptr(v),
                             mcr._ptr(eps), mcr._stream(stream)), "mc3_h_eps")
    return H, v, eps


def adjoint_source(med: Medium3, dL_dH: torch.Tensor, stream=None) -> torch.Tensor:
    """q* = -mu_a dL/dH / dx^3 (``mc3_adjoint_source``)."""
    lib = load()
    mcr._dev_f32(dL_dH, "dL_dH")
    q = torch.empty(med.shape, dtype=torch.float32, device=dL_dH.device)
    mcr._check(lib.mc3_adjoint_source(C.byref(med.c()), mcr._ptr(dL_dH), mcr._ptr(q), mcr._stream(stream)),
               "mc3_adjoint_source")
    return q


def gradient(med: Medium3, coeff: torch.Tensor, coeff_adj: torch.Tensor, dL_dH: torch.Tensor, stream=None,
             dtype=torch.float64):
    """(dL/dmu_a, dL/dmu_s) per voxel (``mc3_gradient`` / ``mc3_gradient_f32``): FP64 sums, the
    results in ``dtype`` (float32 rounds them once)."""
    lib = load()
    for t, n in ((coeff, "coeff"), (coeff_adj, "coeff_adj"), (dL_dH, "dL_dH")):
        mcr._dev_f32(t, n)
    if coeff.shape != coeff_adj.shape:
        raise ValueError("coeff and coeff_adj must match")
    L = int(round(coeff.shape[0] ** 0.5)) - 1
    if (L + 1) ** 2 != coeff.shape[0]:
        raise ValueError("coeff must have (L+1)^2 channels")
    if dtype not in (torch.float64, torch.float32):
        raise TypeError("dtype must be float64 or float32")
    fn, name = (lib.mc3_gradient, "mc3_gradient") if dtype == torch.float64 else (lib.mc3_gradient_f32,
                                                                                 "mc3_gradient_f32")
    d_mua = torch.empty(med.shape, dtype=dtype, device=coeff.device)
    d_mus = torch.empty_like(d_mua)
    mcr._check(fn(C.byref(med.c()), L, mcr._ptr(coeff), mcr._ptr(coeff_adj), mcr._ptr(dL_dH), mcr._ptr(d_mua),
                  mcr._ptr(d_mus), mcr._stream(stream)), name)
    return d_mua, d_mus


def eps(H: torch.Tensor, Hmeas: torch.Tensor, dx: float, stream=None):
    """eps = 1/2 dx^3 sum (Hmeas - H)^2 (FP64) and dL/dH = -dx^3 (Hmeas - H) from a given H (``mc_eps``
    with the voxel volume as the cell measure)."""
    lib = mcr.load()
    mcr._dev_f32(H, "H")
    mcr._dev_f32(Hmeas, "Hmeas")
    if H.shape != Hmeas.shape:
        raise ValueError("H and Hmeas must match")
    v = torch.empty_like(H)
    e = torch.empty((), dtype=torch.float64, device=H.device)
    d32 = C.c_float(dx).value  # the voxel side as the medium struct carries it (FP32)
    mcr._check(lib.mc_eps(H.numel(), d32 * d32 * d32, mcr._ptr(H), mcr._ptr(Hmeas), mcr._ptr(v), mcr._ptr(e),
                          mcr._stream(stream)), "mc_eps")
    return e, v
