"""mc_forward_noalloc: the forward model for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they run the forward model (their device memory is
owned by another allocator or pool, or the synchronisation cudaMalloc implies is not acceptable
in their loop).  mc_forward_noalloc keeps its scratch in a fixed array inside the library.  This
test calls it through the C ABI and checks it against mc_forward, call after call, including a
call of another size in between (the array keeps the previous call's contents), and checks that
oversize problems are refused, that it applies mc_forward's argument rules, and that its device
errors reach the caller through mc_check.  It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1608_05238_gb300 import _build, mcr, workloads
from parity_util import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return mcr.load()


def _case(nz, nx, dx, K, n, seed):
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=seed)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(0.85))
    src = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(nx * dx), z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    run = mcr.Run(K=K, n_packets=n, seed=seed)
    return med, src, run


def _noalloc(lib, med, src, run, out):
    out.fill_(float("nan"))
    stream = torch.cuda.current_stream()
    rc = lib.mc_forward_noalloc(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), C.c_void_p(out.data_ptr()),
                                C.c_void_p(stream.cuda_stream))
    assert rc == mcr.OK, mcr.status_string(rc)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _assert_close(a, ref):
    # the same transport kernel on the same packets with order-independent integer tallies: the
    # two entry points agree bit for bit (a parameter one of them forgot would show here)
    assert np.array_equal(a, ref)


def test_noalloc_matches_mc_forward_on_consecutive_calls(lib):
    A = _case(96, 80, 0.1, 16, 200_003, seed=5)
    B = _case(40, 56, 0.05, 32, 120_001, seed=6)
    ref_a = mcr.forward(*A).double().cpu().numpy()
    ref_b = mcr.forward(*B).double().cpu().numpy()
    out_a = torch.empty((2 * A[2].K + 1,) + A[0].shape, device="cuda")
    out_b = torch.empty((2 * B[2].K + 1,) + B[0].shape, device="cuda")
    torch.cuda.synchronize()
    first = _noalloc(lib, *A, out_a)
    _assert_close(first, ref_a)
    free0 = torch.cuda.mem_get_info()[0]
    other = _noalloc(lib, *B, out_b)
    _assert_close(other, ref_b)
    again = _noalloc(lib, *A, out_a)
    _assert_close(again, ref_a)
    assert np.array_equal(first, again)  # no state carried over from the previous call
    assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken by the later calls


def test_noalloc_angular_point_source(lib):
    """The angular point source (a Sec. 4.1 detector as a source) through the no-allocation call."""
    med, _, run = _case(48, 40, 0.1, 8, 100_001, seed=8)
    src = mcr.Source(kind=mcr.ANGULAR_POINT, x0=f32(1.3), z0=f32(2.2), ang_c=(0.0, 0.0, 0.0, -1.0))
    ref = mcr.forward(med, src, run).double().cpu().numpy()
    out = torch.empty((2 * run.K + 1,) + med.shape, device="cuda")
    _assert_close(_noalloc(lib, med, src, run, out), ref)


def test_noalloc_refuses_oversize_problems(lib):
    med, src, run = _case(512, 512, 0.02, 32, 1000, seed=1)
    out = torch.empty((2 * run.K + 1, 512, 512), device="cuda")
    rc = lib.mc_forward_noalloc(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), C.c_void_p(out.data_ptr()), None)
    assert rc == mcr.ERR_SCRATCH
    assert "scratch" in mcr.status_string(rc)
    med, src, _ = _case(16, 16, 0.1, 4, 10, seed=2)
    big = mcr.Run(K=4, n_packets=(1 << 26) + 1)
    out = torch.empty((9, 16, 16), device="cuda")
    assert lib.mc_forward_noalloc(C.byref(med.c()), C.byref(src.c()), C.byref(big.c()), C.c_void_p(out.data_ptr()),
                                  None) == mcr.ERR_SCRATCH
    assert lib.mc_forward_noalloc(C.byref(med.c()), C.byref(src.c()), C.byref(big.c()), None, None) == mcr.ERR_ARG


def test_noalloc_applies_mc_forward_argument_rules(lib):
    med, src, run = _case(16, 16, 0.1, 4, 1000, seed=3)
    out = torch.empty((9, 16, 16), device="cuda")
    bad = mcr.Run(K=4, n_packets=1000)
    c = bad.c()
    c.accumulate = 2  # mc_forward refuses anything but 0 and 1
    args = (C.byref(med.c()), C.byref(src.c()))
    assert lib.mc_forward_noalloc(*args, C.byref(c), C.c_void_p(out.data_ptr()), None) == mcr.ERR_ARG
    assert lib.mc_forward(*args, C.byref(c), C.c_void_p(out.data_ptr()), None, None) == mcr.ERR_ARG
    m = med.c()
    m.nx, m.nz = 1 << 13, 1 << 13  # 2^26 pixels: beyond the deposit key's range
    assert lib.mc_forward_noalloc(C.byref(m), C.byref(src.c()), C.byref(run.c()), C.c_void_p(out.data_ptr()),
                                  None) == mcr.ERR_ARG


def test_noalloc_device_errors_reach_mc_check(lib):
    try:  # start from a clean latch
        mcr.check()
    except mcr.McrError:
        pass
    # a packet ended by the event cap (dense scatterer, at most 3 flights)
    mua = torch.full((8, 8), 0.001, device="cuda")
    mus = torch.full((8, 8), 50.0, device="cuda")
    med = mcr.Medium(mua, mus, 0.1, 0.0)
    src = mcr.Source(kind=mcr.ISO_POINT, x0=0.4, z0=0.4)
    out = torch.empty((3, 8, 8), device="cuda")
    _noalloc(lib, med, src, mcr.Run(K=1, n_packets=100, max_events=3), out)
    with pytest.raises(mcr.McrError) as e:
        mcr.check()
    assert e.value.status == mcr.ERR_EVENT_LIMIT
    mcr.check()  # reported once, then cleared
    # a negative mu: nothing is deposited, and the error is still reported after a later good call
    bad = mua.clone()
    bad[2, 3] = -1.0
    got = _noalloc(lib, mcr.Medium(bad, mus, 0.1, 0.0), src, mcr.Run(K=1, n_packets=100), out)
    assert not got.any()
    _noalloc(lib, med, src, mcr.Run(K=1, n_packets=100), out)
    with pytest.raises(mcr.McrError) as e:
        mcr.check()
    assert e.value.status == mcr.ERR_MEDIUM
    mcr.check()
