"""Raw fixed-point sums and their finalisation on the GPU (the pieces of packet sharding): the sums of
disjoint packet ranges added together equal the sums of the whole range bit for bit, and
mc_finalize of those sums equals mc_forward / mc_adjoint of the whole range bit for bit."""
import numpy as np
import pytest
import torch

from paper_1608_05238_gb300 import _build, mcr, shard, workloads
from parity_util import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()


def _case(K=16):
    nz, nx, dx = 48, 40, 0.08
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=31)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(0.85))
    src = mcr.Source(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(nx * dx), z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    q = torch.from_numpy((np.random.default_rng(5).normal(size=(nz, nx)) * mua).astype(np.float32)).cuda()
    return med, src, q


@pytest.mark.parametrize("K", [0, 8, 16, 32])
def test_forward_ranges_add_and_finalize_matches_mc_forward(K):
    med, src, _ = _case()
    n, first = 300_001, 12_345
    whole = mcr.forward_raw(med, src, mcr.Run(K=K, n_packets=n, first_packet=first, seed=4))
    parts = mcr.forward_raw(med, src, mcr.Run(K=K, n_packets=100_000, first_packet=first, seed=4))
    mcr.forward_raw(med, src, mcr.Run(K=K, n_packets=n - 100_000, first_packet=first + 100_000, seed=4,
                                      accumulate=True), out=parts)
    assert whole.dtype == torch.int64 and whole.shape == (2 * K + 1,) + med.shape
    assert torch.equal(whole, parts)
    run = mcr.Run(K=K, n_packets=n, first_packet=first, seed=4)
    ref = mcr.forward(med, src, run)
    assert torch.equal(mcr.finalize(med, run, parts, src=src), ref)
    # finalize's accumulate adds the coefficients of a second illumination
    acc = ref.clone()
    mcr.finalize(med, mcr.Run(K=K, n_packets=n, accumulate=True), parts, src=src, out=acc)
    assert torch.equal(acc, ref + ref)
    mcr.check()


@pytest.mark.parametrize("K", [4, 32])
def test_adjoint_ranges_add_and_finalize_matches_mc_adjoint(K):
    med, _, q = _case()
    n = 250_000
    run = mcr.Run(K=K, n_packets=n, seed=8, stream_id=1)
    a = mcr.adjoint_raw(med, q, mcr.Run(K=K, n_packets=90_000, seed=8, stream_id=1))
    mcr.adjoint_raw(med, q, mcr.Run(K=K, n_packets=n - 90_000, first_packet=90_000, seed=8, stream_id=1,
                                    accumulate=True), out=a)
    assert torch.equal(a, mcr.adjoint_raw(med, q, run))
    assert torch.equal(mcr.finalize(med, run, a, qstar=q), mcr.adjoint(med, q, run))
    mcr.check()


def test_single_rank_shard_equals_plain_calls():
    med, src, q = _case()
    run = mcr.Run(K=8, n_packets=200_000, seed=2)
    assert torch.equal(shard.forward(med, src, run), mcr.forward(med, src, run))
    arun = mcr.Run(K=8, n_packets=200_000, seed=3, stream_id=1)
    assert torch.equal(shard.adjoint(med, q, arun), mcr.adjoint(med, q, arun))


def test_raw_calls_refuse_bad_arguments():
    med, src, q = _case()
    with pytest.raises(mcr.McrError):   # more than one launch's packets per raw call
        mcr.forward_raw(med, src, mcr.Run(K=2, n_packets=(1 << 26) + 1))
    with pytest.raises(mcr.McrError):   # the sector tally has no raw form
        mcr.forward_raw(med, src, mcr.Run(K=2, n_packets=10, sectors=8))
    with pytest.raises(ValueError):
        mcr.finalize(med, mcr.Run(K=2, n_packets=10), torch.zeros((5,) + med.shape, dtype=torch.int64,
                                                                     device="cuda"))
