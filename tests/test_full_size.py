"""The 256x256, K = 32 gradient workload at its full size, in the launch configuration the benchmark
times (default launch shape, 1e7 packets): parity on sampled packets the oracle can follow one by
one, and properties that hold at any size (bit reproducibility, packet ranges that add up,
energy bookkeeping, the FP64 gradient combine against the oracle's functionals)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import RunParams
from oracle import functionals as F
from paper_1608_05238_gb300 import _build, mcr, workloads
from parity_util import assert_parity

pytestmark = pytest.mark.gpu

N_FULL = 10_000_000


@pytest.fixture(scope="module")
def setup():
    _build.build()
    mcr.load()
    w = workloads.grad256(N_FULL)
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    med = mcr.Medium(torch.from_numpy(w.mua).cuda(), torch.from_numpy(w.mus).cuda(), dx, g)
    med_t = mcr.Medium(torch.from_numpy(w.mua_true).cuda(), torch.from_numpy(w.mus_true).cuda(), dx, g)
    src = mcr.Source(**w.sources[0])
    Hmeas = mcr.h_eps(med_t, mcr.forward(med_t, src, mcr.Run(K=0, n_packets=1_000_000, seed=1001)))
    return w, med, src, Hmeas


def test_sampled_packets_of_the_full_run_match_the_oracle(setup):
    """Packets 4,990,000 .. 5,009,999 of the 1e7-packet forward run and of an adjoint run (from a
    seeded adjoint source with the workload's structure) on the full grid at K = 32."""
    w, med, src, Hmeas = setup
    dx, g = med.dx, med.g
    mua64, mus64 = w.mua.astype(np.float64), w.mus.astype(np.float64)
    first, n = 4_990_000, 20_000
    run = mcr.Run(K=w.K, n_packets=n, first_packet=first, seed=77)
    G = mcr.forward(med, src, run).double().cpu().numpy()
    O = oracle.forward(mua64, mus64, dx, g, src.as_dict(), RunParams(K=w.K, n_packets=n, first_packet=first, seed=77),
                       with_variance=True)
    assert_parity(G, O.coeff, O.coeff[0], np.sqrt(O.a0_var), label="grad256 forward sample")
    # an adjoint source with this workload's structure, from the inputs alone: q* = -mu_a v / dx^2
    # with v ~ mu_a - mu_a,true (nonzero on the inclusions)
    qn = (-mua64 * (mua64 - w.mua_true.astype(np.float64)) / dx ** 2).astype(np.float32)
    q = torch.from_numpy(qn).cuda()
    arun = mcr.Run(K=w.K, n_packets=n, first_packet=first, seed=78, stream_id=1)
    Ga = mcr.adjoint(med, q, arun).double().cpu().numpy()
    rp = RunParams(K=w.K, n_packets=n, first_packet=first, seed=78, stream_id=1)
    Oa = oracle.adjoint(mua64, mus64, dx, g, qn, rp)
    Oabs = oracle.adjoint(mua64, mus64, dx, g, np.abs(qn), rp, with_variance=True)
    assert_parity(Ga, Oa.coeff, Oabs.coeff[0], np.sqrt(Oabs.a0_var), label="grad256 adjoint sample")


def test_full_run_is_reproducible_splits_and_conserves_energy(setup):
    w, med, src, _ = setup
    full, st = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=N_FULL, seed=9), stats=True)
    again = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=N_FULL, seed=9))
    assert torch.equal(full, again)
    h = N_FULL // 2 + 12_345
    a = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=h, seed=9))
    b = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=N_FULL - h, first_packet=h, seed=9))
    comb = (a.double() * h + b.double() * (N_FULL - h)) / N_FULL
    ref = full.double()
    assert torch.allclose(comb, ref, rtol=2e-6, atol=2e-7 * ref.abs().max().item())
    assert st["launched"] == N_FULL and st["segments"] > 100 * N_FULL
    absorbed = float((med.mua.double() * full[0].double()).sum()) * float(med.dx) ** 2 * N_FULL
    assert abs(absorbed - st["absorbed_w"]) <= 1e-5 * st["launched_w"]
    assert abs(st["launched_w"] + st["rr_net_w"] - st["escaped_w"] - st["killed_w"] - st["absorbed_w"]) \
        <= 1e-9 * st["launched_w"]


def test_full_size_gradient_combine_matches_oracle_functionals(setup):
    """At the full size of one gradient evaluation (256^2 pixels, K = 32: 65 channels), the FP64
    gradient kernel and the H / eps kernel equal the oracle's Eqs. 22/28 and Eq. 2 on the same
    seeded inputs (coefficient tensors of the workload's scale, drawn here, not produced by the
    transport)."""
    w, med, src, Hmeas = setup
    rng = np.random.default_rng(31)
    C, nz, nx = 2 * w.K + 1, w.nz, w.nx
    c = (rng.normal(size=(C, nz, nx)) * 0.1).astype(np.float32)
    c[0] = np.abs(c[0]) * 10
    ca = (rng.normal(size=(C, nz, nx)) * 0.1).astype(np.float32)
    vn = (rng.normal(size=(nz, nx)) * 1e-3).astype(np.float32)
    ga, gs = mcr.gradient(med, torch.from_numpy(c).cuda(), torch.from_numpy(ca).cuda(), torch.from_numpy(vn).cuda())
    ra, rs = F.dL_dmu(c.astype(np.float64), ca.astype(np.float64), vn.astype(np.float64), float(med.dx), float(med.g))
    ga, gs = ga.cpu().numpy(), gs.cpu().numpy()
    assert np.max(np.abs(ga - ra)) <= 1e-12 * np.max(np.abs(ra))
    assert np.max(np.abs(gs - rs)) <= 1e-12 * np.max(np.abs(rs))
    Hm = (w.mua_true * c[0] * 1.1).astype(np.float32)
    H, _, eps = mcr.h_eps(med, torch.from_numpy(c).cuda(), torch.from_numpy(Hm).cuda())
    H32 = (w.mua * c[0]).astype(np.float32)  # one FP32 product
    assert np.array_equal(H.cpu().numpy(), H32)
    e_ref = F.error_functional(Hm.astype(np.float64), H32.astype(np.float64), float(med.dx))
    assert abs(eps.item() - e_ref) <= 1e-12 * e_ref
