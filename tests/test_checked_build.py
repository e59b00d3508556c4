"""The checked build (libmcr_checked.so: every tally, medium and record index range-checked on the
device and every deposit checked for a finite weight; a failed check skips the access and
latches MCR_ERR_CHECK) -- the stand-in for a device memory checker.  The main paths run through it:
forward and adjoint at K = 0, 8, 32 and 64 (incl. the per-lane remainder and the collision merge),
a mixed batch, the sector and time tallies, and the sorted-record deposit; no check may fire, and
every result equals the normal library's bit for bit (the guards do not change the arithmetic)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1608_05238_gb300 import _build, mcr, workloads
from parity_util import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    _build.build()
    return mcr.load(), mcr.load_checked()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _forward(lib, med, src, run, C_):
    out = torch.empty((C_,) + med.shape, device="cuda")
    rc = lib.mc_forward(C.byref(med.c()), C.byref(src.c()), C.byref(run.c()), C.c_void_p(out.data_ptr()), None,
                        _stream())
    assert rc == mcr.OK
    return out


def _adjoint(lib, med, q, run):
    out = torch.empty((2 * run.K + 1,) + med.shape, device="cuda")
    rc = lib.mc_adjoint(C.byref(med.c()), C.c_void_p(q.data_ptr()), C.byref(run.c()), C.c_void_p(out.data_ptr()),
                        None, _stream())
    assert rc == mcr.OK
    return out


def _batch(lib, probs, common, launch):
    arr = (mcr._Problem * len(probs))(*[p.c(common.K) for p in probs])
    ln = mcr._Launch(*launch)
    rc = lib.mc_run_batch(arr, len(probs), C.byref(common.c()), C.byref(ln), None, _stream())
    assert rc == mcr.OK
    return [p.out.clone() for p in probs]


def _clean(lib):
    rc = lib.mc_check(_stream())
    assert rc == mcr.OK, lib.mc_status_string(rc).decode()


def test_checked_library_reports_itself(libs):
    _, chk = libs
    assert b"checked" in chk.mc_version()
    assert b"checked" in chk.mc_status_string(mcr.ERR_CHECK)


@pytest.mark.parametrize("K", [0, 8, 32, 64])
def test_forward_and_adjoint_pass_the_checks_and_match(libs, K):
    lib, chk = libs
    mua, mus = workloads.small_hetero(56, 48, 0.07, seed=K + 3)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(0.07), f32(0.85))
    src = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(48 * 0.07), z1=0.0, dir_x=0.25, dir_z=1.0)
    run = mcr.Run(K=K, n_packets=60_001, seed=K, w_threshold=0.05, roulette_p=0.3)
    a = _forward(chk, med, src, run, 2 * K + 1)
    _clean(chk)
    assert torch.equal(a, _forward(lib, med, src, run, 2 * K + 1))
    q = torch.from_numpy(np.random.default_rng(K).normal(size=(56, 48)).astype(np.float32)).cuda()
    arun = mcr.Run(K=K, n_packets=40_003, seed=K + 1, stream_id=1)
    b = _adjoint(chk, med, q, arun)
    _clean(chk)
    assert torch.equal(b, _adjoint(lib, med, q, arun))


def test_batch_merge_records_sectors_and_time_bins_pass_the_checks(libs):
    lib, chk = libs
    mua, mus = workloads.small_hetero(40, 52, 0.08, seed=2)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(0.08), f32(0.8))
    src = mcr.Source(kind=mcr.ISO_POINT, x0=f32(1.7), z0=f32(1.1))
    q = torch.from_numpy(np.random.default_rng(9).normal(size=(40, 52)).astype(np.float32)).cuda()
    for K in (16, 32):
        probs = [mcr.Problem(med, 30_000, seed=3, source=src), mcr.Problem(med, 25_000, seed=4, stream_id=1, qstar=q)]
        common = mcr.Run(K=K, n_packets=0)
        for launch in ((128, 0, 2, 0, 2, 0, 0), (128, 0, 1, 0, 1, 0, 0)):  # merge + launch order / neither
            got = _batch(chk, probs, common, launch)
            _clean(chk)
            assert all(torch.equal(x, y) for x, y in zip(got, _batch(lib, probs, common, launch)))
        for pr in probs:  # sorted-record deposit, with chunks that overflow and run again directly
            launch = (128, 0, 0, 0, 0, 2, 40_000)
            got = _batch(chk, [pr], common, launch)[0]
            _clean(chk)
            assert torch.equal(got, _batch(lib, [pr], common, (128, 0, 0, 0, 0, 1, 0))[0])
    for run, C_ in ((mcr.Run(K=0, n_packets=30_000, seed=5, sectors=13), 13),
                    (mcr.Run(K=0, n_packets=30_000, seed=5, time_bins=9, time_bin_mm=0.4), 9)):
        got = _forward(chk, med, src, run, C_)
        _clean(chk)
        assert torch.equal(got, _forward(lib, med, src, run, C_))
