"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every symbol that
include/mcr.h declares, and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1608_05238_gb300 import _build, denoise_ops, mcr, mcr3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:mc3?|dn)_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return mcr.load()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for n in ("mc_forward", "mc_adjoint", "mc_gradient", "mc_h_eps", "mc_adjoint_source", "dn_conv", "dn_wgrad",
              "mc3_forward", "mc3_adjoint", "mc3_gradient"):
        assert n in names
    assert set(names) == set(mcr.EXPORTS) | set(mcr.DIAG_EXPORTS) | set(denoise_ops.EXPORTS) | set(mcr3.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for n in _declared_symbols():
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    assert mcr.status_string(0) == "ok"
    assert "argument" in mcr.status_string(mcr.ERR_ARG)
    assert "sm_103a" in mcr.version()
    assert mcr.status_string(12345) == "unknown status"


def _medium(nx=4, nz=3, dx=0.1, g=0.5, mua=1, mus=1):
    # non-null dummy pointers: only the host-side checks run before any CUDA call
    return mcr._Medium(nx, nz, dx, g, mua, mus)


@pytest.mark.parametrize("kw", [dict(nx=0), dict(nz=-1), dict(dx=0.0), dict(dx=float("nan")), dict(g=1.0),
                                dict(g=-1.5), dict(mua=None), dict(mus=None)])
def test_bad_medium_rejected_on_host(lib, kw):
    m = _medium(**kw)
    src = mcr._Source(mcr.PENCIL, 0.1, 0.0, 0, 0, 0.0, 1.0, 1.0)
    run = mcr.Run(K=2, n_packets=10).c()
    assert lib.mc_forward(C.byref(m), C.byref(src), C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc_gradient(C.byref(m), 2, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), None,
                           None) == mcr.ERR_ARG


@pytest.mark.parametrize("kw", [dict(K=-1), dict(K=mcr.MAX_K + 1), dict(roulette_p=0.0), dict(roulette_p=1.5),
                                dict(w_threshold=-1.0), dict(first_packet=2 ** 64 - 5, n_packets=10)])
def test_bad_run_rejected_on_host(lib, kw):
    args = dict(K=2, n_packets=10)
    args.update(kw)
    run = mcr.Run(**args).c()
    m = _medium()
    src = mcr._Source(mcr.PENCIL, 0.1, 0.0, 0, 0, 0.0, 1.0, 1.0)
    assert lib.mc_forward(C.byref(m), C.byref(src), C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc_adjoint(C.byref(m), C.c_void_p(8), C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG


@pytest.mark.parametrize("src", [dict(kind=7), dict(kind=mcr.PENCIL, dir_x=0.0, dir_z=0.0),
                                 dict(kind=mcr.LINE, x0=float("inf")), dict(kind=mcr.ISO_POINT, power=float("nan"))])
def test_bad_source_rejected_on_host(lib, src):
    s = mcr.Source(**src).c()
    run = mcr.Run(K=1, n_packets=10).c()
    assert lib.mc_forward(C.byref(_medium()), C.byref(s), C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG


def test_null_outputs_rejected_on_host(lib):
    run = mcr.Run(K=1, n_packets=10).c()
    src = mcr._Source(mcr.PENCIL, 0.1, 0.0, 0, 0, 0.0, 1.0, 1.0)
    m = _medium()
    assert lib.mc_forward(C.byref(m), C.byref(src), C.byref(run), None, None, None) == mcr.ERR_ARG
    assert lib.mc_forward(C.byref(m), None, C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc_adjoint(C.byref(m), None, C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc_h_eps(C.byref(m), None, None, None, None, None, None) == mcr.ERR_ARG
    # eps requested without H^meas
    assert lib.mc_h_eps(C.byref(m), C.c_void_p(8), None, None, None, C.c_void_p(8), None) == mcr.ERR_ARG
    assert lib.mc_adjoint_source(C.byref(m), None, C.c_void_p(8), None) == mcr.ERR_ARG
    assert lib.mc_gradient(C.byref(m), 1, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), None, None, None) == mcr.ERR_ARG


def test_binding_refuses_cpu_tensors(lib):
    import torch
    med = mcr.Medium(torch.zeros(3, 4), torch.zeros(3, 4), 0.1, 0.5)
    with pytest.raises(TypeError):
        mcr.forward(med, mcr.Source(mcr.PENCIL, x0=0.2), mcr.Run(K=1, n_packets=10))


def _medium3(nx=4, ny=5, nz=3, dx=0.1, g=0.5, mua=1, mus=1):
    return mcr3._Medium3(nx, ny, nz, dx, g, mua, mus)


@pytest.mark.parametrize("kw", [dict(nx=0), dict(ny=-2), dict(nz=0), dict(dx=0.0), dict(dx=float("inf")), dict(g=1.0),
                                dict(g=-1.0), dict(mua=None), dict(mus=None), dict(nx=1024, ny=1024, nz=64)])
def test_bad_medium3_rejected_on_host(lib, kw):
    mcr3.load()
    m = _medium3(**kw)
    src = mcr3.Source3(mcr.PENCIL, 0.1, 0.1, 0.0).c()
    run = mcr.Run(K=2, n_packets=10).c()
    p = C.c_void_p(8)
    assert lib.mc3_forward(C.byref(m), C.byref(src), C.byref(run), p, None, None) == mcr.ERR_ARG
    assert lib.mc3_adjoint(C.byref(m), p, C.byref(run), p, None, None) == mcr.ERR_ARG
    assert lib.mc3_gradient(C.byref(m), 2, p, p, p, p, p, None) == mcr.ERR_ARG
    assert lib.mc3_h_eps(C.byref(m), p, None, p, None, None, None) == mcr.ERR_ARG
    assert lib.mc3_adjoint_source(C.byref(m), p, p, None) == mcr.ERR_ARG


@pytest.mark.parametrize("kw", [dict(K=-1), dict(K=mcr3.MAX_L + 1), dict(sectors=4), dict(roulette_p=0.0),
                                dict(n_packets=2 ** 26 + 1), dict(first_packet=2 ** 64 - 5, n_packets=10)])
def test_bad_run3_rejected_on_host(lib, kw):
    mcr3.load()
    args = dict(K=2, n_packets=10)
    args.update(kw)
    run = mcr.Run(**args).c()
    m = _medium3()
    src = mcr3.Source3(mcr.ISO_POINT, 0.1, 0.1, 0.1).c()
    p = C.c_void_p(8)
    assert lib.mc3_forward(C.byref(m), C.byref(src), C.byref(run), p, None, None) == mcr.ERR_ARG
    assert lib.mc3_adjoint(C.byref(m), p, C.byref(run), p, None, None) == mcr.ERR_ARG


@pytest.mark.parametrize("src", [dict(kind=mcr.LINE), dict(kind=mcr.ANGULAR_POINT), dict(kind=9),
                                 dict(kind=mcr.PENCIL, dir_x=0.0, dir_y=0.0, dir_z=0.0),
                                 dict(kind=mcr.ISO_POINT, y0=float("nan")), dict(kind=mcr.PENCIL, power=float("inf"))])
def test_bad_source3_rejected_on_host(lib, src):
    mcr3.load()
    s = mcr3.Source3(**src).c()
    run = mcr.Run(K=1, n_packets=10).c()
    m = _medium3()
    assert lib.mc3_forward(C.byref(m), C.byref(s), C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc3_forward(C.byref(m), None, C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc3_adjoint(C.byref(m), None, C.byref(run), C.c_void_p(8), None, None) == mcr.ERR_ARG
    assert lib.mc3_gradient(C.byref(m), mcr3.MAX_L + 1, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8),
                            C.c_void_p(8), None) == mcr.ERR_ARG
