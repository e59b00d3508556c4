"""Thin Python binding of libmcr (include/mcr.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module passes torch device pointers, the
current CUDA stream and plain structs through ctypes, and raises :class:`McrError` on a negative
status.  There is no CPU fallback: if ``libmcr.so`` is missing or no GPU is present the calls
raise.  Names follow the paper (Hochuli et al., arXiv 1608.05238): ``mua``/``mus`` are mu_a and
mu_s maps [nz, nx] in 1/mm, ``dx`` the pixel side in mm, ``g`` the 2D Henyey-Greenstein
anisotropy, ``K`` the harmonic order; coefficient tensors are [2K+1, nz, nx] with channel 0 = a_0,
2n-1 = a_n, 2n = b_n.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, field

import torch

from . import _build

PENCIL, LINE, ISO_POINT, ANGULAR_POINT = 0, 1, 2, 3
MAX_K = 64

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_EVENT_LIMIT, ERR_TALLY_OVERFLOW, ERR_MEDIUM = 0, -1, -2, -3, -4, -5, -6
ERR_CHECK = -8  # checked build only

# every symbol declared in include/mcr.h
EXPORTS = ("mc_forward", "mc_forward_noalloc", "mc_adjoint", "mc_forward_raw", "mc_adjoint_raw", "mc_finalize",
           "mc_run_batch", "mc_h_eps", "mc_eps", "mc_dot",
           "mc_adjoint_source", "mc_gradient", "mc_gradient_f32", "mc_check", "mc_last_run_info",
           "mc_release_workspace", "mc_status_string", "mc_version")
# measurement and test entry points (include/mcr_diag.h), not part of the method's interface
DIAG_EXPORTS = ("mc_reduction_probe", "mc_philox_blocks", "dn_wait_probe")
MAX_BATCH = 64
ERR_SCRATCH = -7


class McrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class _Medium(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("dx", C.c_float), ("g", C.c_float),
                ("mua", C.c_void_p), ("mus", C.c_void_p)]


MAX_ANG = 8


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_float), ("z0", C.c_float), ("x1", C.c_float), ("z1", C.c_float),
                ("dir_x", C.c_float), ("dir_z", C.c_float), ("power", C.c_float), ("n_ang", C.c_int32),
                ("ang_c", C.c_float * MAX_ANG), ("ang_s", C.c_float * MAX_ANG)]


class _Run(C.Structure):
    _fields_ = [("K", C.c_int32), ("max_scatter", C.c_uint32), ("n_packets", C.c_uint64),
                ("first_packet", C.c_uint64), ("seed", C.c_uint64), ("stream_id", C.c_uint32),
                ("max_events", C.c_uint32), ("w_threshold", C.c_float), ("roulette_p", C.c_float),
                ("accumulate", C.c_uint32), ("sectors", C.c_uint32), ("time_bins", C.c_uint32),
                ("time_bin_mm", C.c_float)]


class _Problem(C.Structure):
    _fields_ = [("medium", _Medium), ("source", _Source), ("qstar", C.c_void_p), ("n_packets", C.c_uint64),
                ("first_packet", C.c_uint64), ("seed", C.c_uint64), ("stream_id", C.c_uint32), ("coeff", C.c_void_p)]


class _Launch(C.Structure):
    _fields_ = [("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("merge_collisions", C.c_int32),
                ("shared_tally", C.c_int32), ("launch_order", C.c_int32), ("deposit", C.c_int32),
                ("record_capacity", C.c_int64)]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("launched", "flights", "collisions", "segments", "escapes", "rr_kill",
                                          "rr_survive", "scatter_limit", "event_limit")] + \
               [(n, C.c_double) for n in ("launched_w", "escaped_w", "rr_net_w", "killed_w", "absorbed_w")]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libmcr.so (built by ``__graft_entry__.build()`` / ``_build.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libmcr.so is not built ({_build.LIB}); run __graft_entry__.build() first")
        _lib = _declare(C.CDLL(_build.LIB))
        return _lib


_lib_checked = None


def load_checked() -> C.CDLL:
    """The checked build, libmcr_checked.so (the transport library compiled with MCR_CHECKED: every
    tally, medium and record index range-checked on the device, a failed check latching
    ERR_CHECK instead of touching memory).  Same C ABI as libmcr.so minus the denoiser calls."""
    global _lib_checked
    with _lock:
        if _lib_checked is None:
            if not os.path.exists(_build.LIB_CHECKED):
                raise RuntimeError(f"libmcr_checked.so is not built ({_build.LIB_CHECKED})")
            _lib_checked = _declare(C.CDLL(_build.LIB_CHECKED))
        return _lib_checked


def _declare(lib: C.CDLL) -> C.CDLL:
    """Argument and result types of the C ABI on a loaded library."""
    vp = C.c_void_p
    lib.mc_forward.argtypes = [C.POINTER(_Medium), C.POINTER(_Source), C.POINTER(_Run), vp, C.POINTER(_Stats), vp]
    lib.mc_forward_noalloc.argtypes = [C.POINTER(_Medium), C.POINTER(_Source), C.POINTER(_Run), vp, vp]
    lib.mc_adjoint.argtypes = [C.POINTER(_Medium), vp, C.POINTER(_Run), vp, C.POINTER(_Stats), vp]
    lib.mc_forward_raw.argtypes = [C.POINTER(_Medium), C.POINTER(_Source), C.POINTER(_Run), vp,
                                   C.POINTER(_Stats), vp]
    lib.mc_adjoint_raw.argtypes = [C.POINTER(_Medium), vp, C.POINTER(_Run), vp, C.POINTER(_Stats), vp]
    lib.mc_finalize.argtypes = [C.POINTER(_Medium), C.POINTER(_Source), vp, C.POINTER(_Run), vp, vp, vp]
    lib.mc_run_batch.argtypes = [C.POINTER(_Problem), C.c_int32, C.POINTER(_Run), C.POINTER(_Launch),
                                 C.POINTER(_Stats), vp]
    lib.mc_h_eps.argtypes = [C.POINTER(_Medium), vp, vp, vp, vp, vp, vp]
    lib.mc_adjoint_source.argtypes = [C.POINTER(_Medium), vp, vp, vp]
    lib.mc_gradient.argtypes = [C.POINTER(_Medium), C.c_int32, vp, vp, vp, vp, vp, vp]
    lib.mc_gradient_f32.argtypes = [C.POINTER(_Medium), C.c_int32, vp, vp, vp, vp, vp, vp]
    lib.mc_eps.argtypes = [C.c_int64, C.c_double, vp, vp, vp, vp, vp]
    lib.mc_dot.argtypes = [C.c_int64, vp, vp, vp, vp]
    lib.mc_check.argtypes = [vp]
    lib.mc_reduction_probe.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32, vp]
    lib.mc_philox_blocks.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_int32,
                                     C.POINTER(C.c_uint32)]
    lib.mc_philox_blocks.restype = C.c_int
    lib.mc_last_run_info.argtypes = [C.c_int32, C.POINTER(_Stats), C.POINTER(C.c_float)]
    lib.mc_release_workspace.argtypes = []
    lib.mc_status_string.argtypes = [C.c_int]
    lib.mc_status_string.restype = C.c_char_p
    lib.mc_version.argtypes = []
    lib.mc_version.restype = C.c_char_p
    for name in ("mc_forward", "mc_forward_noalloc", "mc_adjoint", "mc_forward_raw", "mc_adjoint_raw",
                 "mc_finalize", "mc_run_batch", "mc_h_eps", "mc_eps", "mc_dot",
                 "mc_adjoint_source", "mc_gradient", "mc_gradient_f32", "mc_check", "mc_last_run_info",
                 "mc_release_workspace"):
        getattr(lib, name).restype = C.c_int
    return lib


def status_string(status: int) -> str:
    return load().mc_status_string(int(status)).decode()


def version() -> str:
    return load().mc_version().decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise McrError(rc, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


@dataclass
class Medium:
    """Pixelised medium (Sec. 3): mu_a, mu_s maps [nz, nx] (float32 CUDA), pixel side dx, HG g."""
    mua: torch.Tensor
    mus: torch.Tensor
    dx: float
    g: float

    @property
    def shape(self):
        return tuple(self.mua.shape)

    def c(self) -> _Medium:
        _dev_f32(self.mua, "mua")
        _dev_f32(self.mus, "mus")
        if self.mua.shape != self.mus.shape or self.mua.dim() != 2:
            raise ValueError("mua and mus must have the same [nz, nx] shape")
        nz, nx = self.mua.shape
        return _Medium(nx, nz, float(self.dx), float(self.g), self.mua.data_ptr(), self.mus.data_ptr())


@dataclass
class Source:
    """Forward source: PENCIL / LINE / ISO_POINT / ANGULAR_POINT (positions in mm, direction normalised
    by the library).  ANGULAR_POINT launches angles theta (from +z) with density
    (1 + sum_n ang_c[n-1] cos n theta + ang_s[n-1] sin n theta) / (2 pi), n <= 8."""
    kind: int
    x0: float = 0.0
    z0: float = 0.0
    x1: float = 0.0
    z1: float = 0.0
    dir_x: float = 0.0
    dir_z: float = 1.0
    power: float = 1.0
    ang_c: tuple = ()
    ang_s: tuple = ()

    def c(self) -> _Source:
        ac, as_ = list(self.ang_c), list(self.ang_s)
        n = max(len(ac), len(as_))
        if n > MAX_ANG:
            raise ValueError(f"at most {MAX_ANG} angular harmonics")
        ac, as_ = ac + [0.0] * (MAX_ANG - len(ac)), as_ + [0.0] * (MAX_ANG - len(as_))
        return _Source(int(self.kind), self.x0, self.z0, self.x1, self.z1, self.dir_x, self.dir_z, self.power, n,
                       (C.c_float * MAX_ANG)(*ac), (C.c_float * MAX_ANG)(*as_))

    def as_dict(self) -> dict:
        return dict(kind=self.kind, x0=self.x0, z0=self.z0, x1=self.x1, z1=self.z1, dir_x=self.dir_x,
                    dir_z=self.dir_z, power=self.power, ang_c=list(self.ang_c), ang_s=list(self.ang_s))


@dataclass
class Run:
    """MC run parameters (mcr_run)."""
    K: int
    n_packets: int
    seed: int = 0
    stream_id: int = 0
    first_packet: int = 0
    max_scatter: int = 0xFFFFFFFF
    max_events: int = 10_000_000
    w_threshold: float = 1e-4
    roulette_p: float = 0.1
    accumulate: bool = False  # add into ``out`` instead of overwriting it
    sectors: int = 0          # > 0 (forward only): discrete-ordinates tally in that many equal sectors
    time_bins: int = 0        # > 0 (forward only): fluence per path-length bin of width time_bin_mm (mm)
    time_bin_mm: float = 0.0

    def c(self) -> _Run:
        return _Run(int(self.K), int(self.max_scatter), int(self.n_packets), int(self.first_packet),
                    int(self.seed) & 0xFFFFFFFFFFFFFFFF, int(self.stream_id), int(self.max_events),
                    float(self.w_threshold), float(self.roulette_p), 1 if self.accumulate else 0,
                    int(self.sectors), int(self.time_bins), float(self.time_bin_mm))


def _stats_dict(st: _Stats) -> dict:
    return {n: getattr(st, n) for n, _ in _Stats._fields_}


def _coeff_out(med: Medium, K: int, out, sectors: int = 0):
    nz, nx = med.shape
    C = sectors if sectors > 0 else 2 * K + 1  # ``sectors``: the channel count of a sector or time tally
    if out is None:
        return torch.empty((C, nz, nx), dtype=torch.float32, device=med.mua.device)
    _dev_f32(out, "out")
    if tuple(out.shape) != (C, nz, nx):
        raise ValueError("out must be [2K+1, nz, nx] (or [sectors, nz, nx])")
    return out


def forward(med: Medium, src: Source, run: Run, out=None, stats: bool = False, stream=None):
    """Forward harmonic radiance MC (``mc_forward``); returns coeff [2K+1, nz, nx] (and stats dict), or
    with ``run.sectors`` = M > 0 the radiance integrated over each of M equal angular sectors
    [m 2pi/M, (m+1) 2pi/M) of theta (from +z), [M, nz, nx] (they sum to a_0), or with
    ``run.time_bins`` = T > 0 the fluence per path-length bin [b w, (b+1) w), w = ``run.time_bin_mm``
    (the last bin open-ended), [T, nz, nx] (they sum to a_0)."""
    lib = load()
    coeff = _coeff_out(med, run.K, out, run.time_bins or run.sectors)
    st = _Stats() if stats else None
    rc = lib.mc_forward(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), _ptr(coeff),
                        C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "mc_forward")
    return (coeff, _stats_dict(st)) if stats else coeff


def adjoint(med: Medium, qstar: torch.Tensor, run: Run, out=None, stats: bool = False, stream=None):
    """Adjoint harmonic radiance MC from q* (``mc_adjoint``); returns coeff_adj (and stats dict)."""
    lib = load()
    _dev_f32(qstar, "qstar")
    if tuple(qstar.shape) != med.shape:
        raise ValueError("qstar must have the medium's shape")
    coeff = _coeff_out(med, run.K, out)
    st = _Stats() if stats else None
    rc = lib.mc_adjoint(C.byref(med.c()), _ptr(qstar), C.byref(run.c()), _ptr(coeff),
                        C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "mc_adjoint")
    return (coeff, _stats_dict(st)) if stats else coeff


# Packets per raw call (mc_forward_raw / mc_adjoint_raw): longer ranges are added call by call.
RAW_MAX_PACKETS = 1 << 26


def _raw_out(med: Medium, K: int, out):
    nz, nx = med.shape
    if out is None:
        return torch.empty((2 * K + 1, nz, nx), dtype=torch.int64, device=med.mua.device)
    if not (out.is_cuda and out.dtype == torch.int64 and out.is_contiguous() and
            tuple(out.shape) == (2 * K + 1, nz, nx)):
        raise TypeError("raw tally must be a contiguous int64 CUDA tensor [2K+1, nz, nx]")
    return out


def forward_raw(med: Medium, src: Source, run: Run, out=None, stats: bool = False, stream=None):
    """Raw 64-bit fixed-point sums of a forward run (``mc_forward_raw``), int64 [2K+1, nz, nx];
    with ``run.accumulate`` added into ``out``.  Sums of disjoint packet ranges add exactly."""
    lib = load()
    tally = _raw_out(med, run.K, out)
    st = _Stats() if stats else None
    rc = lib.mc_forward_raw(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), _ptr(tally),
                            C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "mc_forward_raw")
    return (tally, _stats_dict(st)) if stats else tally


def adjoint_raw(med: Medium, qstar: torch.Tensor, run: Run, out=None, stats: bool = False, stream=None):
    """Raw fixed-point sums of an adjoint run (``mc_adjoint_raw``; odd orders not yet turned)."""
    lib = load()
    _dev_f32(qstar, "qstar")
    if tuple(qstar.shape) != med.shape:
        raise ValueError("qstar must have the medium's shape")
    tally = _raw_out(med, run.K, out)
    st = _Stats() if stats else None
    rc = lib.mc_adjoint_raw(C.byref(med.c()), _ptr(qstar), C.byref(run.c()), _ptr(tally),
                            C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "mc_adjoint_raw")
    return (tally, _stats_dict(st)) if stats else tally


def finalize(med: Medium, run: Run, tally: torch.Tensor, src: Source | None = None, qstar: torch.Tensor | None = None,
             out=None, stream=None) -> torch.Tensor:
    """Coefficients [2K+1, nz, nx] from raw sums (``mc_finalize``): ``run.n_packets`` is the total
    of all ranges in ``tally``; exactly one of ``src`` (forward) and ``qstar`` (adjoint)."""
    lib = load()
    _raw_out(med, run.K, tally)
    if (src is None) == (qstar is None):
        raise ValueError("finalize takes exactly one of src / qstar")
    if qstar is not None:
        _dev_f32(qstar, "qstar")
    coeff = _coeff_out(med, run.K, out)
    rc = lib.mc_finalize(C.byref(med.c()), C.byref(src.c()) if src is not None else None, _ptr(qstar),
                         C.byref(run.c()), _ptr(tally), _ptr(coeff), _stream(stream))
    _check(rc, "mc_finalize")
    return coeff


@dataclass
class Problem:
    """One problem of a batched launch: a forward source (``source``) or an adjoint q* (``qstar``)."""
    medium: Medium
    n_packets: int
    seed: int = 0
    stream_id: int = 0
    first_packet: int = 0
    source: Source | None = None
    qstar: torch.Tensor | None = None
    out: torch.Tensor | None = None

    def c(self, K: int) -> _Problem:
        if (self.source is None) == (self.qstar is None):
            raise ValueError("a problem has exactly one of source / qstar")
        if self.out is None:
            self.out = torch.empty((2 * K + 1,) + self.medium.shape, dtype=torch.float32,
                                   device=self.medium.mua.device)
        _dev_f32(self.out, "out")
        if tuple(self.out.shape) != (2 * K + 1,) + self.medium.shape:
            raise ValueError("out must be [2K+1, nz, nx]")
        if self.qstar is not None:
            _dev_f32(self.qstar, "qstar")
            if tuple(self.qstar.shape) != self.medium.shape:
                raise ValueError("qstar must have the medium's shape")
        src = self.source.c() if self.source is not None else _Source()
        return _Problem(self.medium.c(), src, self.qstar.data_ptr() if self.qstar is not None else None,
                        int(self.n_packets), int(self.first_packet), int(self.seed) & 0xFFFFFFFFFFFFFFFF,
                        int(self.stream_id), self.out.data_ptr())


def run_batch(problems: list, common: Run, launch: tuple | None = None, stats: bool = False, stream=None):
    """All ``problems`` in one persistent transport launch (``mc_run_batch``); returns their outputs.

    ``common`` gives K and the termination parameters; ``launch`` = (threads_per_block,
    blocks_per_sm[, merge_collisions[, shared_tally[, launch_order]]]) or None for the defaults
    (0 in a field: its default; merge_collisions 1 off, 2 on; shared_tally 2: per-block
    shared-memory tally where it applies; launch_order 1 off, 2 on: packets in the order of their
    launch position; deposit 1 direct, 2 sorted records (a batch of one harmonic problem);
    record_capacity: records per chunk of the sorted-record deposit).  The call can be captured in a CUDA graph once a
    first call has grown the library's workspace to this batch's size.
    """
    lib = load()
    if not 1 <= len(problems) <= MAX_BATCH:
        raise ValueError(f"1..{MAX_BATCH} problems per batch")
    arr = (_Problem * len(problems))(*[p.c(common.K) for p in problems])
    ln = _Launch(*launch) if launch is not None else None
    st = _Stats() if stats else None
    rc = lib.mc_run_batch(arr, len(problems), C.byref(common.c()), C.byref(ln) if ln is not None else None,
                          C.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "mc_run_batch")
    outs = [p.out for p in problems]
    return (outs, _stats_dict(st)) if stats else outs


def h_eps(med: Medium, coeff: torch.Tensor, Hmeas: torch.Tensor | None = None, stream=None):
    """H = mu_a a_0; with Hmeas also dL/dH = -dx^2 (Hmeas - H) and eps (``mc_h_eps``).

    Returns H, or (H, dL_dH, eps) with eps a 0-d float64 CUDA tensor.
    """
    lib = load()
    _dev_f32(coeff, "coeff")
    H = torch.empty(med.shape, dtype=torch.float32, device=coeff.device)
    if Hmeas is None:
        _check(lib.mc_h_eps(C.byref(med.c()), _ptr(coeff), None, _ptr(H), None, None, _stream(stream)), "mc_h_eps")
        return H
    _dev_f32(Hmeas, "Hmeas")
    v = torch.empty_like(H)
    eps = torch.empty((), dtype=torch.float64, device=coeff.device)
    _check(lib.mc_h_eps(C.byref(med.c()), _ptr(coeff), _ptr(Hmeas), _ptr(H), _ptr(v), _ptr(eps), _stream(stream)),
           "mc_h_eps")
    return H, v, eps


def adjoint_source(med: Medium, dL_dH: torch.Tensor, stream=None) -> torch.Tensor:
    """q* = -mu_a dL/dH / dx^2 (``mc_adjoint_source``)."""
    lib = load()
    _dev_f32(dL_dH, "dL_dH")
    q = torch.empty(med.shape, dtype=torch.float32, device=dL_dH.device)
    _check(lib.mc_adjoint_source(C.byref(med.c()), _ptr(dL_dH), _ptr(q), _stream(stream)), "mc_adjoint_source")
    return q


def gradient(med: Medium, coeff: torch.Tensor, coeff_adj: torch.Tensor, dL_dH: torch.Tensor, stream=None,
             dtype=torch.float64):
    """(dL/dmu_a, dL/dmu_s) per pixel (``mc_gradient`` / ``mc_gradient_f32``, Eqs. 22 and 28 x dx^2).

    The sums run in FP64 either way; ``dtype`` float32 rounds the results once on output.
    """
    lib = load()
    for t, n in ((coeff, "coeff"), (coeff_adj, "coeff_adj"), (dL_dH, "dL_dH")):
        _dev_f32(t, n)
    K = (coeff.shape[0] - 1) // 2
    if coeff.shape != coeff_adj.shape:
        raise ValueError("coeff and coeff_adj must match")
    d_mua = torch.empty(med.shape, dtype=dtype, device=coeff.device)
    d_mus = torch.empty_like(d_mua)
    fn, name = (lib.mc_gradient, "mc_gradient") if dtype == torch.float64 else (lib.mc_gradient_f32, "mc_gradient_f32")
    if dtype not in (torch.float64, torch.float32):
        raise TypeError("dtype must be float64 or float32")
    _check(fn(C.byref(med.c()), K, _ptr(coeff), _ptr(coeff_adj), _ptr(dL_dH), _ptr(d_mua), _ptr(d_mus),
              _stream(stream)), name)
    return d_mua, d_mus


def eps(H: torch.Tensor, Hmeas: torch.Tensor, dx: float, stream=None):
    """eps = 1/2 dx^2 sum (Hmeas - H)^2 (FP64) and dL/dH = -dx^2 (Hmeas - H) from a given H (``mc_eps``)."""
    lib = load()
    _dev_f32(H, "H")
    _dev_f32(Hmeas, "Hmeas")
    if H.shape != Hmeas.shape:
        raise ValueError("H and Hmeas must match")
    v = torch.empty_like(H)
    e = torch.empty((), dtype=torch.float64, device=H.device)
    d32 = C.c_float(dx).value  # the pixel side as the medium struct carries it (FP32)
    _check(lib.mc_eps(H.numel(), d32 * d32, _ptr(H), _ptr(Hmeas), _ptr(v), _ptr(e), _stream(stream)), "mc_eps")
    return e, v


def dot(a: torch.Tensor, b: torch.Tensor, stream=None) -> torch.Tensor:
    """sum a_i b_i of two float32 CUDA tensors of equal size in FP64, fixed order (``mc_dot``);
    returns a 0-d float64 CUDA tensor."""
    _dev_f32(a, "a")
    _dev_f32(b, "b")
    if a.numel() != b.numel():
        raise ValueError("a and b must have the same number of elements")
    out = torch.empty((), dtype=torch.float64, device=a.device)
    _check(load().mc_dot(a.numel(), _ptr(a), _ptr(b), _ptr(out), _stream(stream)), "mc_dot")
    return out


def check(stream=None):
    """Synchronise and raise any latched device error (``mc_check``)."""
    _check(load().mc_check(_stream(stream)), "mc_check")


def last_run_info(which: str = "forward"):
    """(stats dict, transport kernel ms) of the last forward / adjoint / batch call (``mc_last_run_info``)."""
    st = _Stats()
    ms = C.c_float(0.0)
    code = {"forward": 0, "adjoint": 1, "batch": 2}[which]
    _check(load().mc_last_run_info(code, C.byref(st), C.byref(ms)), "mc_last_run_info")
    return _stats_dict(st), float(ms.value)


def release_workspace():
    _check(load().mc_release_workspace(), "mc_release_workspace")


def philox_blocks(counters, keys):
    """Philox4x32-10 blocks from the transport's device function (``mc_philox_blocks``):
    ``counters`` [n][4] and ``keys`` [n][2] 32-bit words in, [n][4] words out (a list of tuples)."""
    n = len(counters)
    if n != len(keys) or n < 1:
        raise ValueError("one key per counter, at least one")
    ctr = (C.c_uint32 * (4 * n))(*[int(w) & 0xFFFFFFFF for c in counters for w in c])
    key = (C.c_uint32 * (2 * n))(*[int(w) & 0xFFFFFFFF for k in keys for w in k])
    out = (C.c_uint32 * (4 * n))()
    _check(load().mc_philox_blocks(ctr, key, n, out), "mc_philox_blocks")
    return [tuple(out[4 * i:4 * i + 4]) for i in range(n)]


def reduction_probe(tally: torch.Tensor, n_coeff: int, iters: int, blocks: int, threads: int = 256, stream=None):
    """``mc_reduction_probe``: (blocks x threads / 32) warps each add 1 to the first n_coeff words of
    ``iters`` pseudo-random rows of ``tally`` (int64 [rows, row_words], device) in the deposit's
    32-lane coalesced pattern -- the ceiling of the tally reductions, timed by the caller."""
    assert tally.is_cuda and tally.dtype == torch.int64 and tally.dim() == 2 and tally.is_contiguous()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = load().mc_reduction_probe(C.c_void_p(tally.data_ptr()), tally.shape[0], tally.shape[1], n_coeff, iters,
                                   blocks, threads, C.c_void_p(s.cuda_stream))
    if rc != 0:
        raise McrError(rc, "mc_reduction_probe")
