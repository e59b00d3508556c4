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
    """Packets 4,990,000 .. 5,009,999 of the 1e7-packet forward run and of the adjoint run (from
    the q* of this workload) on the full grid at K = 32."""
    w, med, src, Hmeas = setup
    dx, g = med.dx, med.g
    mua64, mus64 = w.mua.astype(np.float64), w.mus.astype(np.float64)
    first, n = 4_990_000, 20_000
    run = mcr.Run(K=w.K, n_packets=n, first_packet=first, seed=77)
    G = mcr.forward(med, src, run).double().cpu().numpy()
    O = oracle.forward(mua64, mus64, dx, g, src.as_dict(), RunParams(K=w.K, n_packets=n, first_packet=first, seed=77),
                       with_variance=True)
    assert_parity(G, O.coeff, O.coeff[0], np.sqrt(O.a0_var), label="grad256 forward sample")
    # the adjoint source of this workload, from a 1e6-packet forward estimate
    coeff = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=1_000_000, seed=5))
    _, v, _ = mcr.h_eps(med, coeff, Hmeas)
    q = mcr.adjoint_source(med, v)
    arun = mcr.Run(K=w.K, n_packets=n, first_packet=first, seed=78, stream_id=1)
    Ga = mcr.adjoint(med, q, arun).double().cpu().numpy()
    qn = q.cpu().numpy()
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
    """On the full-size coefficient tensors of one gradient evaluation (1e7 + 1e7 packets), the
    FP64 gradient kernel equals the oracle's Eqs. 22/28 evaluated on the same inputs."""
    w, med, src, Hmeas = setup
    coeff = mcr.forward(med, src, mcr.Run(K=w.K, n_packets=N_FULL, seed=11))
    H, v, eps = mcr.h_eps(med, coeff, Hmeas)
    q = mcr.adjoint_source(med, v)
    adj = mcr.adjoint(med, q, mcr.Run(K=w.K, n_packets=N_FULL, seed=12, stream_id=1))
    ga, gs = mcr.gradient(med, coeff, adj, v)
    c, ca = coeff.double().cpu().numpy(), adj.double().cpu().numpy()
    vn = v.double().cpu().numpy()
    ra, rs = F.dL_dmu(c, ca, vn, float(med.dx), float(med.g))
    ga, gs = ga.cpu().numpy(), gs.cpu().numpy()
    assert np.max(np.abs(ga - ra)) <= 1e-12 * np.max(np.abs(ra))
    assert np.max(np.abs(gs - rs)) <= 1e-12 * np.max(np.abs(rs))
    e_ref = F.error_functional(Hmeas.double().cpu().numpy(), H.double().cpu().numpy(), float(med.dx))
    assert abs(eps.item() - e_ref) <= 1e-12 * e_ref
