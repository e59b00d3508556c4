"""GPU parity of the 3D form (spherical-harmonic tallies, Sec. 3.1's named extension) through the
C ABI (include/mcr3.h) against the FP64 3D oracle on identical Philox streams.

Tolerances are those of the 2D parity tests (parity_util), with the absolute tally A taken as
sqrt(2L+1) |c_00| of |W| packets: every real harmonic obeys |Y_lm| <= sqrt((2l+1) / 4 pi), so a
packet's |c_lm| contribution is at most sqrt(2l+1) times its c_00 contribution.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import RunParams
from oracle import functionals as F
from paper_1608_05238_gb300 import _build, mcr, mcr3, workloads
from parity_util import assert_parity, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr3.load()
    yield
    torch.cuda.synchronize()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _orc_run(run: mcr.Run) -> RunParams:
    return RunParams(K=run.K, n_packets=run.n_packets, seed=run.seed, stream_id=run.stream_id,
                     first_packet=run.first_packet, max_scatter=run.max_scatter, max_events=run.max_events,
                     w_threshold=run.w_threshold, roulette_p=run.roulette_p)


def _forward_case(mua, mus, dx, g, src, run, label):
    dx, g = f32(dx), f32(g)
    src = {k: (f32(v) if isinstance(v, (float, np.floating)) else v) for k, v in src.items()}
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    G, st = mcr3.forward(med, mcr3.Source3(**src), run, stats=True)
    G = G.double().cpu().numpy()
    O = oracle.forward3(mua.astype(np.float64), mus.astype(np.float64), dx, g, src, _orc_run(run),
                        with_variance=True)
    s = math.sqrt(2 * run.K + 1)
    info = assert_parity(G, O.coeff, s * O.coeff[0], s * np.sqrt(O.a0_var), label=label)
    assert st["launched"] == O.stats["launched"] == run.n_packets
    return G, O, st, info


def test_forward3_pencil_L2_ragged():
    mua, mus = workloads.small_hetero3(16, 20, 24, 0.1, seed=1)
    src = dict(kind=mcr.PENCIL, x0=1.23, y0=0.97, z0=0.0, dir_x=0.0, dir_y=0.0, dir_z=1.0, power=1.0)
    _forward_case(mua, mus, 0.1, 0.9, src, mcr.Run(K=2, n_packets=200_003, seed=7), "3D pencil L2")


def test_forward3_iso_point_L5_oblique_grid():
    """36 channels: two warp passes per voxel deposit; a non-cubic grid."""
    mua, mus = workloads.small_hetero3(13, 21, 17, 0.08, seed=2)
    src = dict(kind=mcr.ISO_POINT, x0=0.731, y0=0.913, z0=0.517, power=2.5)
    _forward_case(mua, mus, 0.08, 0.75, src, mcr.Run(K=5, n_packets=150_017, seed=11, stream_id=3), "3D iso L5")


def test_forward3_oblique_pencil_L8():
    """81 channels: three warp passes; an oblique pencil (direction normalised by the library)."""
    mua, mus = workloads.small_hetero3(14, 12, 18, 0.1, seed=3)
    d = np.array([0.6, 0.2, 1.1]) / np.linalg.norm([0.6, 0.2, 1.1])  # the oracle takes a unit vector
    src = dict(kind=mcr.PENCIL, x0=0.4, y0=0.3, z0=0.0, dir_x=d[0], dir_y=d[1], dir_z=d[2], power=1.0)
    run = mcr.Run(K=8, n_packets=100_019, seed=5, w_threshold=0.8, roulette_p=0.3)
    G, O, st, _ = _forward_case(mua, mus, 0.1, 0.8, src, run, "3D oblique pencil L8")
    assert st["rr_kill"] > 0 and st["rr_survive"] > 0


def _adjoint_case(mua, mus, dx, g, q, run, label):
    dx, g = f32(dx), f32(g)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    G, st = mcr3.adjoint(med, _dev(q), run, stats=True)
    G = G.double().cpu().numpy()
    m64, s64 = mua.astype(np.float64), mus.astype(np.float64)
    O = oracle.adjoint3(m64, s64, dx, g, q, _orc_run(run))
    Oabs = oracle.volume3(m64, s64, dx, g, np.abs(q), _orc_run(run), adjoint=False, with_variance=True)
    s = math.sqrt(2 * run.K + 1)
    assert_parity(G, O.coeff, s * Oabs.coeff[0], s * np.sqrt(Oabs.a0_var), label=label)
    assert st["launched"] == run.n_packets
    assert st["launched_w"] == O.stats["launched_w"]
    return G, O


def test_adjoint3_signed_source_L4():
    mua, mus = workloads.small_hetero3(12, 14, 16, 0.1, seed=4)
    rng = np.random.default_rng(3)
    q = (rng.normal(size=mua.shape) * (rng.uniform(size=mua.shape) < 0.3)).astype(np.float32)
    _adjoint_case(mua, mus, 0.1, 0.8, q, mcr.Run(K=4, n_packets=150_001, seed=21, stream_id=1), "3D adjoint L4")


def test_adjoint3_single_voxel_L3_is_the_turned_forward_run():
    """From one voxel, the adjoint coefficients are (-1)^l times those of the same packets tallied
    forward: the oracle's non-adjoint run of the same source, turned here."""
    mua, mus = workloads.small_hetero3(10, 10, 10, 0.1, seed=5)
    q = np.zeros(mua.shape, np.float32)
    q[4, 6, 3] = -2.0
    run = mcr.Run(K=3, n_packets=100_000, seed=9)
    G, O = _adjoint_case(mua, mus, 0.1, 0.9, q, run, "3D adjoint voxel")
    fwd = oracle.volume3(mua.astype(np.float64), mus.astype(np.float64), f32(0.1), f32(0.9), q, _orc_run(run),
                         adjoint=False).coeff
    for c in range(16):
        assert np.allclose(O.coeff[c], (-1) ** math.isqrt(c) * fwd[c], rtol=1e-12, atol=0)


def test_gradient3_h_eps_and_adjoint_source_match_the_functionals():
    """mc3_gradient / mc3_h_eps / mc3_adjoint_source against the oracle functionals on the SAME
    seeded inputs (no transport; each kernel is fed numpy arrays, never another kernel's output):
    FP64 sums in the same channel order."""
    rng = np.random.default_rng(9)
    L, nz, ny, nx, dx, g = 6, 9, 11, 13, f32(0.05), f32(0.85)
    C = (L + 1) ** 2
    c = rng.normal(size=(C, nz, ny, nx)).astype(np.float32)
    cs = rng.normal(size=(C, nz, ny, nx)).astype(np.float32)
    c[0] = np.abs(c[0])
    mua = rng.uniform(0.01, 0.5, (nz, ny, nx)).astype(np.float32)
    mus = rng.uniform(1.0, 9.0, (nz, ny, nx)).astype(np.float32)
    Hm = rng.uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    H, v, eps = mcr3.h_eps(med, _dev(c), _dev(Hm))
    H, v = H.double().cpu().numpy(), v.double().cpu().numpy()
    Href = F.absorbed_energy3(mua, c)
    assert np.allclose(H, Href, rtol=2e-6, atol=0)
    # dL/dH and eps from the oracle's own H: they differ from the kernel's by its FP32 rounding of H
    vref = F.dL_dH_eps3(Hm, Href, dx)
    assert np.max(np.abs(v - vref)) <= 1e-6 * dx ** 3 * np.abs(Href).max()
    assert abs(eps.item() - F.error_functional3(Hm, Href, dx)) <= 1e-5 * eps.item()
    H_only = mcr3.h_eps(med, _dev(c)).double().cpu().numpy()
    assert np.array_equal(H_only, H)
    vin = rng.normal(size=(nz, ny, nx)).astype(np.float32)  # dL/dH input of the next two kernels
    q = mcr3.adjoint_source(med, _dev(vin)).double().cpu().numpy()
    assert np.allclose(q, F.adjoint_source3(mua, vin, dx), rtol=2e-6, atol=0)
    ga, gs = mcr3.gradient(med, _dev(c), _dev(cs), _dev(vin))
    wa, ws = F.dL_dmu3(c, cs, vin, dx, g)
    assert np.allclose(ga.cpu().numpy(), wa, rtol=1e-12, atol=1e-12 * np.abs(wa).max())
    assert np.allclose(gs.cpu().numpy(), ws, rtol=1e-12, atol=1e-12 * np.abs(ws).max())


def test_beer_lambert_column_closed_form():
    """No scattering, a pencil down the axis of a voxel column: c_l0 in voxel k of the column is
    e^{-sum_{j<k} mu_a dx} (1 - e^{-mu_a dx}) / mu_a sqrt((2l+1) / 4 pi) / dx^3 and every other
    coefficient (and voxel) is 0."""
    nz, ny, nx, dx, L = 12, 3, 3, f32(0.25), 4
    mua = np.random.default_rng(1).uniform(0.1, 1.5, (nz, ny, nx)).astype(np.float32)
    mus = np.zeros_like(mua)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, 0.0)
    src = mcr3.Source3(mcr.PENCIL, x0=f32(0.375), y0=f32(0.375), z0=0.0, dir_z=1.0)
    G = mcr3.forward(med, src, mcr.Run(K=L, n_packets=4096, seed=1)).double().cpu().numpy()
    want = np.zeros_like(G)
    T = 1.0
    for k in range(nz):
        a = float(mua[k, 1, 1])
        t = T * (1 - math.exp(-a * dx)) / a / dx ** 3
        for l in range(L + 1):
            want[l * l + l, k, 1, 1] = t * math.sqrt((2 * l + 1) / (4 * math.pi))
        T *= math.exp(-a * dx)
    assert np.allclose(G, want, rtol=2e-5, atol=1e-6 * np.abs(want).max())


def test_energy_bookkeeping_and_reproducibility():
    """launched + roulette gain = absorbed + escaped + killed, the absorbed weight equals
    sum mu_a Phi V N_p from the GPU's own coefficients, a rerun is bit-identical, and two
    accumulated halves of the packet range average to the whole run."""
    mua, mus = workloads.small_hetero3(10, 12, 14, 0.1, seed=6)
    dx, g = f32(0.1), f32(0.7)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    src = mcr3.Source3(mcr.ISO_POINT, x0=0.61, y0=0.55, z0=0.43)
    N = 400_000
    run = mcr.Run(K=3, n_packets=N, seed=4, w_threshold=0.3, roulette_p=0.5)
    c1, st = mcr3.forward(med, src, run, stats=True)
    assert abs(st["launched_w"] + st["rr_net_w"] - st["absorbed_w"] - st["escaped_w"] - st["killed_w"]) < 1e-9 * N
    phi = math.sqrt(4 * math.pi) * c1[0].double().cpu().numpy()
    absorbed = float(np.sum(mua.astype(np.float64) * phi)) * dx ** 3 * N
    assert abs(absorbed - st["absorbed_w"]) < 2e-5 * st["absorbed_w"]
    c2 = mcr3.forward(med, src, run)
    assert torch.equal(c1, c2)
    half = mcr.Run(K=3, n_packets=N // 2, seed=4, w_threshold=0.3, roulette_p=0.5)
    acc = mcr3.forward(med, src, half)
    half2 = mcr.Run(K=3, n_packets=N // 2, first_packet=N // 2, seed=4, w_threshold=0.3, roulette_p=0.5,
                    accumulate=True)
    mcr3.forward(med, src, half2, out=acc)
    assert torch.allclose(acc / 2, c1, rtol=1e-5, atol=1e-6 * c1.abs().max().item())


def test_device_side_errors():
    """A negative mu_a is refused on the device (MCR_ERR_MEDIUM); an all-zero adjoint source
    launches nothing and gives zero coefficients."""
    mua, mus = workloads.small_hetero3(6, 6, 6, 0.1, seed=7)
    bad = mua.copy()
    bad[2, 3, 1] = -0.1
    med = mcr3.Medium3(_dev(bad), _dev(mus), 0.1, 0.5)
    with pytest.raises(mcr.McrError) as e:
        mcr3.forward(med, mcr3.Source3(mcr.ISO_POINT, 0.3, 0.3, 0.3), mcr.Run(K=1, n_packets=1000))
    assert e.value.status == mcr.ERR_MEDIUM
    med = mcr3.Medium3(_dev(mua), _dev(mus), 0.1, 0.5)
    z = mcr3.adjoint(med, torch.zeros((6, 6, 6), device="cuda"), mcr.Run(K=2, n_packets=1000))
    assert torch.count_nonzero(z).item() == 0
    ok = mcr3.forward(med, mcr3.Source3(mcr.ISO_POINT, 0.3, 0.3, 0.3), mcr.Run(K=1, n_packets=1000))
    assert torch.isfinite(ok).all() and ok[0].sum().item() > 0
    mcr.release_workspace()  # frees the 3D workspace too; the next call allocates it again
    again = mcr3.forward(med, mcr3.Source3(mcr.ISO_POINT, 0.3, 0.3, 0.3), mcr.Run(K=1, n_packets=1000))
    assert torch.equal(again, ok)


def test_gradient3_through_the_gpu_path_matches_the_oracle_gradient():
    """The whole 3D gradient chain on the GPU (forward, H, dL/dH, q*, adjoint, combine) against
    the oracle's chain on the same streams: the maps agree to the tallies' parity tolerance."""
    n, Lside = 10, 0.6
    dx = f32(Lside / n)
    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    mua = (0.15 + 0.1 * np.sin(3 * X) * np.cos(2 * Z) + 0.05 * np.cos(5 * Y)).astype(np.float32)
    mus = (3.0 + 1.0 * np.cos(4 * X + Z - Y)).astype(np.float32)
    Hm = (mua * 1.3).astype(np.float32)
    g, L = f32(0.8), 4
    src = dict(kind=mcr.PENCIL, x0=f32(0.33), y0=f32(0.27), z0=0.0, dir_x=0.0, dir_y=0.0, dir_z=1.0, power=1.0)
    fwd = mcr.Run(K=L, n_packets=300_000, seed=3)
    adj = mcr.Run(K=L, n_packets=300_000, seed=1003, stream_id=1)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    cg = mcr3.forward(med, mcr3.Source3(**src), fwd)
    H, v, _ = mcr3.h_eps(med, cg, _dev(Hm))
    q = mcr3.adjoint_source(med, v)
    ca = mcr3.adjoint(med, q, adj)
    ga, gs = mcr3.gradient(med, cg, ca, v)
    m64, s64 = mua.astype(np.float64), mus.astype(np.float64)
    Fc = oracle.forward3(m64, s64, dx, g, src, _orc_run(fwd)).coeff
    vo = F.dL_dH_eps3(Hm, F.absorbed_energy3(mua, Fc), dx)
    qo = F.adjoint_source3(mua, vo, dx).astype(np.float32)
    A = oracle.adjoint3(m64, s64, dx, g, qo, _orc_run(adj)).coeff
    wa, ws = F.dL_dmu3(Fc, A, vo, dx, g)
    for got, want in ((ga.cpu().numpy(), wa), (gs.cpu().numpy(), ws)):
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 5e-3 * scale
        assert np.abs(got - want).sum() <= 1e-3 * np.abs(want).sum()


def test_grad3d_full_size_sample_and_full_run_properties():
    """The 96^3, L = 4 workload of the 3D benchmark on its full grid: packets 4,900,000 ..
    5,099,999 of a forward and an adjoint run against the oracle (2e5 packets, so that one packet
    whose FP32 and FP64 paths part stays well inside the 1e-4 relative L1 bound), and a
    1e7-packet forward run that is bit reproducible and whose two halves accumulate to it."""
    mua, mus, mua_true, src = workloads.phantom3(96, 0.1, seed=0)
    dx, g, L = f32(0.1), f32(0.9), 4
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    s3 = mcr3.Source3(**src)
    first, n = 4_900_000, 200_000
    run = mcr.Run(K=L, n_packets=n, first_packet=first, seed=77)
    G = mcr3.forward(med, s3, run).double().cpu().numpy()
    m64, s64 = mua.astype(np.float64), mus.astype(np.float64)
    rp = RunParams(K=L, n_packets=n, first_packet=first, seed=77, n_threads=8)
    O = oracle.forward3(m64, s64, dx, g, src, rp, with_variance=True)
    s = math.sqrt(2 * L + 1)
    # grazing segments (along a face or through an edge) that the FP32 and FP64 paths cut
    # differently: voxels only the GPU enters are held to a share of the total, and visited ones
    # get an allowance of 1e-3 of one packet's chord (a full chord adds dx / (N_p dx^3) to c_00)
    chord = s * dx / (n * dx ** 3)
    assert_parity(G, O.coeff, s * O.coeff[0], s * np.sqrt(O.a0_var), label="grad3d forward sample",
                  unvisited_share=1e-7, floor=1e-3 * chord, outliers=(1e-4, 1e-7))
    # an adjoint source with this workload's structure, from the inputs alone: q* = -mu_a v / dx^3
    # with v ~ mu_a - mu_a,true (nonzero on the absorbing spheres)
    qn = (-m64 * (m64 - mua_true.astype(np.float64)) / dx ** 3).astype(np.float32)
    q = _dev(qn)
    arun = mcr.Run(K=L, n_packets=n, first_packet=first, seed=78, stream_id=1)
    Ga = mcr3.adjoint(med, q, arun).double().cpu().numpy()
    rpa = RunParams(K=L, n_packets=n, first_packet=first, seed=78, stream_id=1, n_threads=8)
    Oa = oracle.adjoint3(m64, s64, dx, g, qn, rpa)
    Oabs = oracle.volume3(m64, s64, dx, g, np.abs(qn), rpa, adjoint=False, with_variance=True)
    assert_parity(Ga, Oa.coeff, s * Oabs.coeff[0], s * np.sqrt(Oabs.a0_var), label="grad3d adjoint sample",
                  unvisited_share=1e-7, floor=1e-3 * chord * Oabs.source_strength, outliers=(1e-4, 1e-7))
    # the full forward run: reproducible, and its halves add up
    N = 10_000_000
    full = mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N, seed=9))
    assert torch.equal(full, mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N, seed=9)))
    acc = mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N // 2, seed=9))
    mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N // 2, first_packet=N // 2, seed=9, accumulate=True), out=acc)
    assert torch.allclose(acc / 2, full, rtol=1e-5, atol=1e-6 * full.abs().max().item())


@pytest.mark.parametrize("n_packets", [0, 1, 31, 33])
def test_degenerate_and_ragged_3d(n_packets):
    """A single voxel, L = 0, and packet counts of 0, 1, 31, 33 (empty, one lane, a partial warp,
    one warp plus one) against the oracle; no packets gives zero coefficients and no launches."""
    mua = np.array([[[0.7]]], np.float32)
    mus = np.array([[[3.0]]], np.float32)
    dx, g = f32(0.5), f32(0.6)
    src = dict(kind=mcr.ISO_POINT, x0=f32(0.21), y0=f32(0.33), z0=f32(0.17), power=1.0)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    for L in (0, 2):
        run = mcr.Run(K=L, n_packets=n_packets, seed=4)
        G, st = mcr3.forward(med, mcr3.Source3(**src), run, stats=True)
        assert st["launched"] == n_packets
        if n_packets == 0:
            assert torch.count_nonzero(G).item() == 0
            continue
        O = oracle.forward3(mua.astype(np.float64), mus.astype(np.float64), dx, g, src, _orc_run(run))
        assert np.allclose(G.double().cpu().numpy(), O.coeff, rtol=2e-5, atol=1e-6 * np.abs(O.coeff).max())


def test_maximum_packets_per_call_3d():
    """2^26 packets, the most one call takes, on a small strongly absorbing grid: the tallies do
    not overflow, the bookkeeping closes, and the fluence matches a run of 2^20 packets."""
    mua = np.full((4, 4, 4), 5.0, np.float32)
    mus = np.full((4, 4, 4), 5.0, np.float32)
    med = mcr3.Medium3(_dev(mua), _dev(mus), f32(0.25), f32(0.5))
    src = mcr3.Source3(mcr.ISO_POINT, x0=f32(0.55), y0=f32(0.45), z0=f32(0.6))
    N = 1 << 26
    c, st = mcr3.forward(med, src, mcr.Run(K=2, n_packets=N, seed=6), stats=True)
    assert st["launched"] == N
    assert abs(st["launched_w"] + st["rr_net_w"] - st["absorbed_w"] - st["escaped_w"] - st["killed_w"]) < 1e-9 * N
    small = mcr3.forward(med, src, mcr.Run(K=2, n_packets=1 << 20, seed=7))
    phi, phi_s = c[0].double(), small[0].double()
    assert torch.allclose(phi, phi_s, rtol=0.02, atol=0.02 * phi.max().item())


def test_autograd_3d_equals_the_explicit_chain():
    """HFromMu3 + EpsFromH3: the backward pass is the explicit chain (forward, eps, q*, adjoint,
    FP32 combine) on the same seeds, bit for bit, kept or recomputed; mc3_gradient_f32 is the FP64
    combine rounded once; eps and dL/dH match mc3_h_eps."""
    from paper_1608_05238_gb300.autograd import EpsFromH3, HFromMu3, MCSpec3
    mua, mus = workloads.small_hetero3(10, 11, 12, 0.1, seed=8)
    dx, g = f32(0.1), f32(0.8)
    src = mcr3.Source3(mcr.ISO_POINT, x0=0.61, y0=0.52, z0=0.43)
    Hm = _dev(mua * 0.7)
    med = mcr3.Medium3(_dev(mua), _dev(mus), dx, g)
    grads = []
    for recompute in (False, True):
        spec = MCSpec3(dx=dx, g=g, source=src, L=3, n_packets=200_000, seed=5, adjoint_seed=6, recompute=recompute)
        a, s = _dev(mua).requires_grad_(), _dev(mus).requires_grad_()
        e = EpsFromH3.apply(HFromMu3.apply(a, s, spec), Hm, dx)
        e.backward()
        grads.append((a.grad.clone(), s.grad.clone(), e.item()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
    c = mcr3.forward(med, src, mcr.Run(K=3, n_packets=200_000, seed=5))
    H, v, eps = mcr3.h_eps(med, c, Hm)
    assert abs(eps.item() - grads[0][2]) <= 1e-12 * abs(eps.item())
    ca = mcr3.adjoint(med, mcr3.adjoint_source(med, v), mcr.Run(K=3, n_packets=200_000, seed=6, stream_id=1))
    ga32, gs32 = mcr3.gradient(med, c, ca, v, dtype=torch.float32)
    assert torch.equal(ga32, grads[0][0]) and torch.equal(gs32, grads[0][1])
    ga, gs = mcr3.gradient(med, c, ca, v)
    assert torch.equal(ga.float(), ga32) and torch.equal(gs.float(), gs32)
    e2, v2 = mcr3.eps(H, Hm, dx)
    assert torch.equal(v2, v) and abs(e2.item() - eps.item()) <= 1e-12 * abs(eps.item())
