"""FP64 CPU oracle for the forward/adjoint harmonic radiance Monte Carlo (Hochuli, Powell,
Arridge & Cox, arXiv 1608.05238): the 2D method and the 3D spherical-harmonic form Sec. 3.1 names.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
statement of what the method computes; the CUDA library is checked against
it.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline and
``--impl reference`` legs of ``bench.py`` may import or call anything here.  It shares no code with the
CUDA path: the transport lives in ``mcr_oracle.c`` (plain C, FP64), the
pixelwise functionals (H, epsilon, gradients) in :mod:`oracle.functionals`
(numpy, FP64).

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_pins.py``, ``tests/test_oracle_pins3.py`` and ``tests/test_oracle_gradients.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcr_oracle.c")
_LIB = os.path.join(_HERE, "libmcr_oracle.so")
_lock = threading.Lock()
_lib = None

PENCIL, LINE, ISO_POINT, ANGULAR_POINT = 0, 1, 2, 3
MAX_ANG = 8


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/libmcr_oracle.so`` (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-shared", "-fPIC",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Medium(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double), ("g", C.c_double),
                ("mua", C.POINTER(C.c_double)), ("mus", C.POINTER(C.c_double))]


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_double), ("z0", C.c_double), ("x1", C.c_double),
                ("z1", C.c_double), ("dir_x", C.c_double), ("dir_z", C.c_double), ("power", C.c_double),
                ("n_ang", C.c_int32), ("ang_c", C.c_double * MAX_ANG), ("ang_s", C.c_double * MAX_ANG)]


class _Run(C.Structure):
    _fields_ = [("K", C.c_int32), ("n_threads", C.c_int32), ("n_packets", C.c_uint64),
                ("first_packet", C.c_uint64), ("seed", C.c_uint64), ("stream_id", C.c_uint32),
                ("max_scatter", C.c_uint32), ("max_events", C.c_uint32), ("w_threshold", C.c_double),
                ("roulette_p", C.c_float), ("sectors", C.c_uint32), ("fixed_q", C.c_int32), ("fixed", C.c_uint32),
                ("time_bins", C.c_uint32), ("time_bin_mm", C.c_double)]


class _Medium3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double), ("g", C.c_double),
                ("mua", C.POINTER(C.c_double)), ("mus", C.POINTER(C.c_double))]


class _Source3(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dir_x", C.c_double), ("dir_y", C.c_double), ("dir_z", C.c_double), ("power", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("launched", "flights", "collisions", "segments", "escapes",
                                          "rr_kill", "rr_survive", "scatter_limit", "event_limit")] + \
               [(n, C.c_double) for n in ("launched_w", "escaped_w", "rr_net_w", "absorbed_w", "killed_w")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_forward_raw.argtypes = [C.POINTER(_Medium), C.POINTER(_Source), C.POINTER(_Run),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_Stats)]
            lib.orc_forward_raw.restype = C.c_int
            lib.orc_volume_raw.argtypes = [C.POINTER(_Medium), C.POINTER(C.c_float), C.POINTER(_Run), C.c_int,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_Stats),
                                           C.POINTER(C.c_double)]
            lib.orc_volume_raw.restype = C.c_int
            lib.orc3_forward_raw.argtypes = [C.POINTER(_Medium3), C.POINTER(_Source3), C.POINTER(_Run),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_Stats)]
            lib.orc3_forward_raw.restype = C.c_int
            lib.orc3_volume_raw.argtypes = [C.POINTER(_Medium3), C.POINTER(C.c_float), C.POINTER(_Run), C.c_int,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_Stats),
                                            C.POINTER(C.c_double)]
            lib.orc3_volume_raw.restype = C.c_int
            lib.orc3_sh.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
            lib.orc3_sh.restype = None
            lib.orc3_hg_cos.argtypes = [C.c_double, C.c_double]
            lib.orc3_hg_cos.restype = C.c_double
            lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            lib.orc_philox4x32_10.restype = None
            lib.orc_hg_angle.argtypes = [C.c_double, C.c_double]
            lib.orc_hg_angle.restype = C.c_double
            lib.orc_hg_phase.argtypes = [C.c_double, C.c_double]
            lib.orc_hg_phase.restype = C.c_double
            lib.orc_volume_pick.argtypes = [C.POINTER(C.c_float), C.c_int64, C.c_uint64, C.c_uint32, C.c_uint64]
            lib.orc_volume_pick.restype = C.c_int64
            _lib = lib
    return _lib


@dataclass
class RunParams:
    """Per-run knobs shared by the forward and adjoint oracles."""
    K: int
    n_packets: int
    seed: int = 0
    stream_id: int = 0
    first_packet: int = 0
    max_scatter: int = 0xFFFFFFFF
    max_events: int = 10_000_000
    w_threshold: float = 1e-4
    roulette_p: float = 0.1
    n_threads: int = 0
    sectors: int = 0   # > 0: discrete-ordinates tally in that many equal sectors instead of harmonics
    fixed_q: int | None = None  # set: every deposit term rounded to a multiple of 2^-fixed_q (integer sums)
    time_bins: int = 0          # > 0 (2D forward): fluence per path-length bin of width time_bin_mm
    time_bin_mm: float = 0.0


@dataclass
class Result:
    coeff: np.ndarray        # [2K+1, nz, nx] normalised radiance coefficients (a0, a1, b1, ...)
    a0_var: np.ndarray | None  # [nz, nx] sample variance of the a0 estimate (same normalisation)
    stats: dict
    source_strength: float


def _medium(mua, mus, dx, g):
    mua = np.ascontiguousarray(mua, dtype=np.float64)
    mus = np.ascontiguousarray(mus, dtype=np.float64)
    assert mua.shape == mus.shape and mua.ndim == 2
    m = _Medium(mua.shape[1], mua.shape[0], float(dx), float(g),
                mua.ctypes.data_as(C.POINTER(C.c_double)), mus.ctypes.data_as(C.POINTER(C.c_double)))
    return m, (mua, mus)


def _run(p: RunParams):
    nt = p.n_threads or (os.cpu_count() or 1)
    nt = max(1, min(nt, max(1, p.n_packets)))
    return _Run(p.K, nt, p.n_packets, p.first_packet, p.seed, p.stream_id, p.max_scatter, p.max_events,
                p.w_threshold, p.roulette_p, p.sectors, int(p.fixed_q or 0), 1 if p.fixed_q is not None else 0,
                p.time_bins, p.time_bin_mm)


def _stats_dict(st: _Stats) -> dict:
    return {n: getattr(st, n) for n, _ in _Stats._fields_}


def _finish(raw, sq, n_packets, S, dx, st, sectors=0, volume_power=2) -> Result:
    """Normalised coefficients: harmonics a_0, a_n, b_n, or with ``sectors`` > 0 the angular
    integrals of the radiance over each sector (they sum to a_0); in 3D (``volume_power`` 3) the
    spherical-harmonic coefficients per unit voxel volume.  The variance is that of channel 0's
    per-packet track-weight sums (the fluence estimate up to the constant of channel 0)."""
    A = dx ** volume_power
    norm = S / (n_packets * A) if n_packets > 0 else 0.0
    coeff = raw * norm
    var = None
    if sq is not None and n_packets > 1:
        # a0 = (S/A) mean_p X_p with X_p the per-packet track-weight sum in the pixel;
        # its variance is (S/A)^2 Var(X) / N_p with the unbiased Var(X).
        mean = (raw.sum(axis=0) if sectors else raw[0]) / n_packets
        var = np.maximum(sq / n_packets - mean * mean, 0.0) / (n_packets - 1) * (S / A) ** 2
    return Result(coeff, var, _stats_dict(st), S)


def _source(source: dict) -> _Source:
    ac, as_ = list(source.get("ang_c", ())), list(source.get("ang_s", ()))
    n_ang = max(len(ac), len(as_))
    if n_ang > MAX_ANG:
        raise ValueError(f"at most {MAX_ANG} angular harmonics")
    ac, as_ = ac + [0.0] * (MAX_ANG - len(ac)), as_ + [0.0] * (MAX_ANG - len(as_))
    return _Source(int(source["kind"]), float(source.get("x0", 0.0)), float(source.get("z0", 0.0)),
                   float(source.get("x1", 0.0)), float(source.get("z1", 0.0)), float(source.get("dir_x", 0.0)),
                   float(source.get("dir_z", 1.0)), float(source.get("power", 1.0)), n_ang,
                   (C.c_double * MAX_ANG)(*map(float, ac)), (C.c_double * MAX_ANG)(*map(float, as_)))


def forward_sums(mua, mus, dx, g, source: dict, run: RunParams) -> np.ndarray:
    """Unnormalised tally sums of a forward run over packets [first_packet, first_packet + n_packets),
    [2K+1, nz, nx].  With ``run.fixed_q`` set every deposit term is rounded to a multiple of
    2^-fixed_q, and the sums are returned as int64 in units of that quantum: then the sums of
    disjoint packet ranges add up exactly to the sums of their union."""
    lib = _load()
    m, keep = _medium(mua, mus, dx, g)
    s = _source(source)
    nz, nx = keep[0].shape
    raw = np.zeros((run.time_bins or run.sectors or 2 * run.K + 1, nz, nx), dtype=np.float64)
    st = _Stats()
    rc = lib.orc_forward_raw(C.byref(m), C.byref(s), C.byref(_run(run)), raw.ctypes.data_as(C.POINTER(C.c_double)),
                             None, C.byref(st))
    if rc != 0:
        raise ValueError(f"oracle forward: status {rc}")
    if run.fixed_q is None:
        return raw
    assert np.abs(raw).max() < 2.0 ** 53, "fixed-point sums beyond FP64's exact integers"
    return raw.astype(np.int64)


def forward(mua, mus, dx, g, source: dict, run: RunParams, with_variance: bool = False) -> Result:
    """Forward harmonic radiance MC (Sec. 3, 3.1) from a pencil, line, isotropic or angular point source.

    ``source``: dict(kind=PENCIL|LINE|ISO_POINT|ANGULAR_POINT, x0, z0, x1, z1, dir_x, dir_z, power=1,
    ang_c=[c_1..], ang_s=[s_1..]); an angular point source launches directions theta (from +z)
    with density (1 + sum_n c_n cos n theta + s_n sin n theta) / (2 pi) -- a detector's angular
    sensitivity as a source (Sec. 4.1).
    Returns coefficients a_0, a_n, b_n (Eqs. 9-11) normalised by power / (N_p dx^2).
    """
    lib = _load()
    m, keep = _medium(mua, mus, dx, g)
    ac, as_ = list(source.get("ang_c", ())), list(source.get("ang_s", ()))
    n_ang = max(len(ac), len(as_))
    if n_ang > MAX_ANG:
        raise ValueError(f"at most {MAX_ANG} angular harmonics")
    ac, as_ = ac + [0.0] * (MAX_ANG - len(ac)), as_ + [0.0] * (MAX_ANG - len(as_))
    s = _Source(int(source["kind"]), float(source.get("x0", 0.0)), float(source.get("z0", 0.0)),
                float(source.get("x1", 0.0)), float(source.get("z1", 0.0)), float(source.get("dir_x", 0.0)),
                float(source.get("dir_z", 1.0)), float(source.get("power", 1.0)), n_ang,
                (C.c_double * MAX_ANG)(*map(float, ac)), (C.c_double * MAX_ANG)(*map(float, as_)))
    nz, nx = keep[0].shape
    Cc = run.time_bins or run.sectors or 2 * run.K + 1
    raw = np.zeros((Cc, nz, nx), dtype=np.float64)
    sq = np.zeros((nz, nx), dtype=np.float64) if with_variance else None
    st = _Stats()
    rc = lib.orc_forward_raw(C.byref(m), C.byref(s), C.byref(_run(run)),
                             raw.ctypes.data_as(C.POINTER(C.c_double)),
                             sq.ctypes.data_as(C.POINTER(C.c_double)) if sq is not None else None, C.byref(st))
    if rc != 0:
        raise ValueError(f"oracle forward: status {rc}")
    return _finish(raw, sq, run.n_packets, s.power, dx, st, run.sectors or run.time_bins)


def volume(mua, mus, dx, g, q, run: RunParams, adjoint: bool = True, with_variance: bool = False) -> Result:
    """MC from the signed volumetric isotropic source ``q`` ([nz, nx] float32, per unit area and angle).

    ``adjoint=True`` is the adjoint model of Sec. 4 / Sec. 6: the tally is taken at theta + pi, so
    the result holds the adjoint coefficients a*_n, b*_n.  ``adjoint=False`` tallies at theta (a
    plain forward run from a volumetric source).
    """
    lib = _load()
    m, keep = _medium(mua, mus, dx, g)
    q = np.ascontiguousarray(q, dtype=np.float32)
    nz, nx = keep[0].shape
    assert q.shape == (nz, nx)
    Cc = run.time_bins or run.sectors or 2 * run.K + 1
    raw = np.zeros((Cc, nz, nx), dtype=np.float64)
    sq = np.zeros((nz, nx), dtype=np.float64) if with_variance else None
    st = _Stats()
    S = C.c_double(0.0)
    rc = lib.orc_volume_raw(C.byref(m), q.ctypes.data_as(C.POINTER(C.c_float)), C.byref(_run(run)),
                            1 if adjoint else 0, raw.ctypes.data_as(C.POINTER(C.c_double)),
                            sq.ctypes.data_as(C.POINTER(C.c_double)) if sq is not None else None,
                            C.byref(st), C.byref(S))
    if rc != 0:
        raise ValueError(f"oracle volume: status {rc}")
    return _finish(raw, sq, run.n_packets, S.value, dx, st, run.sectors or run.time_bins)


def adjoint(mua, mus, dx, g, qstar, run: RunParams, with_variance: bool = False) -> Result:
    """Adjoint harmonic radiance MC (Sec. 4, Sec. 6) from q* (per unit area and unit angle)."""
    return volume(mua, mus, dx, g, qstar, run, adjoint=True, with_variance=with_variance)


def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key (Salmon et al., SC'11)."""
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def u01(words) -> np.ndarray:
    """Map 32-bit words to the uniforms ((x >> 9) + 1/2) 2^-23 used by both paths."""
    w = np.asarray(words, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def hg_angle(g: float, u) -> np.ndarray:
    """Scattering angle of Eq. 7 for uniforms ``u`` (vectorised over u)."""
    lib = _load()
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([lib.orc_hg_angle(float(g), float(v)) for v in u])


def hg_phase(g: float, dtheta) -> np.ndarray:
    """2D Henyey-Greenstein phase function of Eq. 6."""
    lib = _load()
    d = np.atleast_1d(np.asarray(dtheta, dtype=np.float64))
    return np.array([lib.orc_hg_phase(float(g), float(v)) for v in d])


def volume_pick(q, seed: int, stream_id: int, packet: int) -> int:
    """Flat pixel index that the volumetric sampler draws for packet ``packet``."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float32)
    return int(lib.orc_volume_pick(q.ctypes.data_as(C.POINTER(C.c_float)), q.size, seed, stream_id, packet))


# ---------------------------------------------------------------------------------------------- 3D
def _medium3(mua, mus, dx, g):
    mua = np.ascontiguousarray(mua, dtype=np.float64)
    mus = np.ascontiguousarray(mus, dtype=np.float64)
    assert mua.shape == mus.shape and mua.ndim == 3
    m = _Medium3(mua.shape[2], mua.shape[1], mua.shape[0], float(dx), float(g),
                 mua.ctypes.data_as(C.POINTER(C.c_double)), mus.ctypes.data_as(C.POINTER(C.c_double)))
    return m, (mua, mus)


def sh3(L: int, sx: float, sy: float, sz: float) -> np.ndarray:
    """Orthonormal real spherical harmonics Y_lm(s), l <= L, at index l^2 + l + m (the 3D basis)."""
    Y = np.zeros((L + 1) ** 2)
    _load().orc3_sh(L, sx, sy, sz, Y.ctypes.data_as(C.POINTER(C.c_double)))
    return Y


def hg3_cos(g: float, u: float) -> float:
    """Cosine of a 3D Henyey-Greenstein scattering angle drawn by the inverse CDF at u."""
    return _load().orc3_hg_cos(g, u)


def forward3(mua, mus, dx, g, source: dict, run: RunParams, with_variance: bool = False) -> Result:
    """3D forward radiance MC (the paper's named 3D extension): voxels [nz, ny, nx], source
    dict(kind=PENCIL|ISO_POINT, x0, y0, z0, dir_x, dir_y, dir_z, power=1), spherical-harmonic
    coefficients c_lm up to l = run.K, [(K+1)^2, nz, ny, nx], normalised by power / (N_p dx^3)."""
    lib = _load()
    m, keep = _medium3(mua, mus, dx, g)
    s = _Source3(int(source["kind"]), float(source.get("x0", 0.0)), float(source.get("y0", 0.0)),
                 float(source.get("z0", 0.0)), float(source.get("dir_x", 0.0)), float(source.get("dir_y", 0.0)),
                 float(source.get("dir_z", 1.0)), float(source.get("power", 1.0)))
    shape = keep[0].shape
    raw = np.zeros(((run.K + 1) ** 2,) + shape, dtype=np.float64)
    sq = np.zeros(shape, dtype=np.float64) if with_variance else None
    st = _Stats()
    rc = lib.orc3_forward_raw(C.byref(m), C.byref(s), C.byref(_run(run)), raw.ctypes.data_as(C.POINTER(C.c_double)),
                              sq.ctypes.data_as(C.POINTER(C.c_double)) if sq is not None else None, C.byref(st))
    if rc != 0:
        raise ValueError(f"oracle forward3: status {rc}")
    return _finish(raw, sq, run.n_packets, s.power, dx, st, volume_power=3)


def volume3(mua, mus, dx, g, q, run: RunParams, adjoint: bool = True, with_variance: bool = False) -> Result:
    """3D run from the signed volumetric isotropic source q ([nz, ny, nx] float32, per unit volume
    and solid angle); ``adjoint=True`` tallies at -s (coefficients c*_lm)."""
    lib = _load()
    m, keep = _medium3(mua, mus, dx, g)
    q = np.ascontiguousarray(q, dtype=np.float32)
    assert q.shape == keep[0].shape
    raw = np.zeros(((run.K + 1) ** 2,) + q.shape, dtype=np.float64)
    sq = np.zeros(q.shape, dtype=np.float64) if with_variance else None
    st = _Stats()
    S = C.c_double(0.0)
    rc = lib.orc3_volume_raw(C.byref(m), q.ctypes.data_as(C.POINTER(C.c_float)), C.byref(_run(run)),
                             1 if adjoint else 0, raw.ctypes.data_as(C.POINTER(C.c_double)),
                             sq.ctypes.data_as(C.POINTER(C.c_double)) if sq is not None else None, C.byref(st),
                             C.byref(S))
    if rc != 0:
        raise ValueError(f"oracle volume3: status {rc}")
    return _finish(raw, sq, run.n_packets, S.value, dx, st, volume_power=3)


def adjoint3(mua, mus, dx, g, qstar, run: RunParams, with_variance: bool = False) -> Result:
    """3D adjoint radiance MC from q* (per unit volume and solid angle)."""
    return volume3(mua, mus, dx, g, qstar, run, adjoint=True, with_variance=with_variance)
