"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical streams.

Sizes are ones the oracle finishes in seconds, spanning many warps' worth of packets and a
ragged tail (packet counts that are not multiples of 32), on square and non-square grids, for
every deposit width (K = 8, 16, 32, 64 -> 1, 2, 3, 5 warp passes per pixel).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import RunParams
from oracle import functionals as F
from paper_1608_05238_gb300 import _build, mcr, workloads
from parity_util import assert_parity, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()
    yield
    torch.cuda.synchronize()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _gpu_forward(mua, mus, dx, g, src, run, stats=False):
    med = mcr.Medium(_dev(mua), _dev(mus), dx, g)
    out = mcr.forward(med, mcr.Source(**src), run, stats=stats)
    if stats:
        c, st = out
        return c.double().cpu().numpy(), st
    return out.double().cpu().numpy()


def _orc_run(run: mcr.Run) -> RunParams:
    return RunParams(K=run.K, n_packets=run.n_packets, seed=run.seed, stream_id=run.stream_id,
                     first_packet=run.first_packet, max_scatter=run.max_scatter, max_events=run.max_events,
                     w_threshold=run.w_threshold, roulette_p=run.roulette_p)


def _src32(src):
    return {k: (f32(v) if isinstance(v, float) else v) for k, v in src.items()}


def _forward_case(mua, mus, dx, g, src, run, label):
    dx, g = f32(dx), f32(g)
    src = _src32(src)
    G, st = _gpu_forward(mua, mus, dx, g, src, run, stats=True)
    O = oracle.forward(mua.astype(np.float64), mus.astype(np.float64), dx, g, src, _orc_run(run),
                       with_variance=True)
    info = assert_parity(G, O.coeff, O.coeff[0], np.sqrt(O.a0_var), label=label)
    assert st["launched"] == O.stats["launched"] == run.n_packets
    return G, O, st, info


def test_forward_pencil32_config():
    """The 32x32 pencil-beam workload in full: K = 8, 1e5 packets, seed 0."""
    w = workloads.pencil32()
    run = mcr.Run(K=w.K, n_packets=w.n_packets, seed=w.seed)
    _forward_case(w.mua, w.mus, w.dx, w.g, w.sources[0], run, "pencil32")


def test_forward_line_heterogeneous_K32_ragged():
    mua, mus = workloads.small_hetero(48, 64, 0.1, seed=3)
    src = dict(kind=mcr.LINE, x0=0.0, z0=0.0, x1=6.4, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    run = mcr.Run(K=32, n_packets=60_001, seed=7)
    _forward_case(mua, mus, 0.1, 0.9, src, run, "line K32")


def test_forward_iso_point_K64_oblique_grid():
    mua, mus = workloads.small_hetero(30, 41, 0.07, seed=4)
    src = dict(kind=mcr.ISO_POINT, x0=1.234, z0=0.987, power=2.5)
    run = mcr.Run(K=64, n_packets=30_017, seed=11, stream_id=3)
    _forward_case(mua, mus, 0.07, 0.75, src, run, "iso K64")


@pytest.mark.parametrize("ac,as_", [([0.0, 0.0, 0.0, -1.0], []), ([0.3, -0.2], [0.25, 0.0, 0.125])])
def test_forward_angular_point_source_K16(ac, as_):
    """A point source with an angular density (the form of a Sec. 4.1 detector) against the oracle:
    the launch angle is the FP32 bisection root of the density's integral on the GPU and the FP64
    one in the oracle, so the streams agree to the FP32 resolution of the angle."""
    mua, mus = workloads.small_hetero(36, 44, 0.08, seed=6)
    src = dict(kind=mcr.ANGULAR_POINT, x0=1.77, z0=1.31, ang_c=ac, ang_s=as_, power=1.5)
    run = mcr.Run(K=16, n_packets=50_003, seed=13, stream_id=5)
    _forward_case(mua, mus, 0.08, 0.8, src, run, "angular point K16")


def test_angular_point_launch_moments_and_rejected_density():
    """Launch directions on the GPU follow the density: with every packet absorbed in the source
    pixel, that pixel's a_n / a_0, b_n / a_0 are the means of cos n theta, sin n theta, whose
    expectations are c_n / 2, s_n / 2.  A density with negative values is refused."""
    n, dx, K, N = 5, 1.0, 6, 1_000_000
    mua, mus = np.full((n, n), 1000.0, np.float32), np.zeros((n, n), np.float32)
    ac, as_ = [0.3, 0.0, 0.2], [0.0, -0.4]
    c = _gpu_forward(mua, mus, dx, 0.0, dict(kind=mcr.ANGULAR_POINT, x0=2.5, z0=2.5, ang_c=ac, ang_s=as_),
                     mcr.Run(K=K, n_packets=N, seed=3))
    a0 = c[0][2, 2]
    sig = 0.75 / math.sqrt(N)
    for m in range(1, K + 1):
        cm = ac[m - 1] if m <= len(ac) else 0.0
        sm = as_[m - 1] if m <= len(as_) else 0.0
        assert abs(c[2 * m - 1][2, 2] / a0 - cm / 2) < 5 * sig, m
        assert abs(c[2 * m][2, 2] / a0 - sm / 2) < 5 * sig, m
    with pytest.raises(mcr.McrError):
        _gpu_forward(mua, mus, dx, 0.0, dict(kind=mcr.ANGULAR_POINT, x0=2.5, z0=2.5, ang_c=[2.0]),
                     mcr.Run(K=1, n_packets=10, seed=3))


def test_reciprocity_case2_odd_detector_gpu():
    """Case 2 (Eqs. 15, 18) on the GPU at 16 x the oracle pin's packets: the detected signal of an
    odd angular detector at r_d from an isotropic source at r_s equals the fluence at r_s of a run
    from r_d with the detector's density turned by pi (the adjoint's theta + pi reading)."""
    nz = nx = 48
    dx, g, K = 0.125, 0.5, 2
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=9)
    ps, pd = (24, 24), (24, 36)
    centre = lambda p: dict(x0=(p[1] + 0.5) * dx, z0=(p[0] + 0.5) * dx)
    det, rec = [], []
    for k in range(4):
        f = _gpu_forward(mua, mus, dx, g, dict(kind=mcr.ISO_POINT, **centre(ps)), mcr.Run(K=K, n_packets=1_000_000,
                                                                                         seed=40 + k))
        det.append(f[0][pd] + f[2][pd])  # (1 + sin theta) / (2 pi): a_0 + b_1
        a = _gpu_forward(mua, mus, dx, g, dict(kind=mcr.ANGULAR_POINT, **centre(pd), ang_s=[-1.0]),
                         mcr.Run(K=0, n_packets=1_000_000, seed=60 + k))
        rec.append(a[0][ps])
    det, rec = np.array(det), np.array(rec)
    se = math.sqrt(det.var(ddof=1) / 4 + rec.var(ddof=1) / 4)
    assert abs(det.mean() - rec.mean()) < 4 * se + 0.01 * det.mean(), (det.mean(), rec.mean(), se)


def test_reciprocity_case3_distributed_source_odd_detector_gpu():
    """Case 3 (Eqs. 16, 19) on the GPU: a distributed isotropic source P_s (unit power; the
    volumetric source q = P_s / (2 pi)) and an odd point detector (1 + sin theta) / (2 pi) at r_d.
    The forward radiance of a volumetric isotropic source is the adjoint run of the same source
    with order n turned back by (-1)^n, so the detected signal is (a*_0 - b*_1)(r_d) of mc_adjoint;
    by reciprocity it equals sum_i dx^2 P_s,i Phi*_i, Phi* the fluence of a run from r_d with the
    detector's density turned by pi (sin theta -> -sin theta)."""
    nz = nx = 48
    dx, g, K = 0.125, 0.5, 2
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=13)
    pd = (24, 36)
    iz, ix = np.mgrid[0:nz, 0:nx]
    Ps = np.exp(-((iz - 24) ** 2 + (ix - 16) ** 2) / (2.0 * 3.0 ** 2))
    Ps /= Ps.sum() * f32(dx) ** 2
    q = (Ps / (2 * math.pi)).astype(np.float32)
    med = mcr.Medium(_dev(mua), _dev(mus), f32(dx), f32(g))
    centre = dict(x0=(pd[1] + 0.5) * dx, z0=(pd[0] + 0.5) * dx)
    det, rec = [], []
    for k in range(4):
        a = mcr.adjoint(med, _dev(q), mcr.Run(K=K, n_packets=1_000_000, seed=80 + k, stream_id=1))
        a = a.double().cpu().numpy()
        det.append(a[0][pd] - a[2][pd])  # forward b_1 = (-1)^1 b*_1
        phi = _gpu_forward(mua, mus, dx, g, dict(kind=mcr.ANGULAR_POINT, **centre, ang_s=[-1.0]),
                           mcr.Run(K=0, n_packets=1_000_000, seed=90 + k))[0]
        rec.append(float((Ps * phi).sum() * f32(dx) ** 2))
    det, rec = np.array(det), np.array(rec)
    se = math.sqrt(det.var(ddof=1) / 4 + rec.var(ddof=1) / 4)
    assert abs(det.mean() - rec.mean()) < 4 * se + 0.01 * det.mean(), (det.mean(), rec.mean(), se)


@pytest.mark.parametrize("M", [8, 37])
def test_forward_sector_tally_parity(M):
    """The discrete-ordinates tally (Sec. 3.1's alternative basis) against the oracle on the same
    streams: one sector per flight from the direction angle (FP32 atan2 on the GPU, FP64 in the
    oracle), one reduction per segment."""
    mua, mus = workloads.small_hetero(40, 52, 0.08, seed=12)
    src = dict(kind=mcr.LINE, x0=0.4, z0=0.0, x1=3.6, z1=0.0, dir_x=0.3, dir_z=1.0)
    run = mcr.Run(K=0, n_packets=40_001, seed=17, sectors=M)
    dx, g = f32(0.08), f32(0.85)
    src = _src32(src)
    G = _gpu_forward(mua, mus, dx, g, src, run)
    O = oracle.forward(mua.astype(np.float64), mus.astype(np.float64), dx, g, src,
                       RunParams(K=0, n_packets=run.n_packets, seed=run.seed, sectors=M))
    assert G.shape == O.coeff.shape == (M, 40, 52)
    # per sector, relative L1 over the field (a packet whose angle sits within FP32 rounding of
    # a sector edge may land in the neighbour on one side)
    for m in range(M):
        assert np.abs(G[m] - O.coeff[m]).sum() <= 2e-3 * np.abs(O.coeff[m]).sum() + 1e-12, m
    # the sectors partition the fluence deposits: their sum is the K = 0 run's a_0
    a0 = _gpu_forward(mua, mus, dx, g, src, mcr.Run(K=0, n_packets=40_001, seed=17))[0]
    assert np.allclose(G.sum(axis=0), a0, rtol=2e-6, atol=1e-9 * a0.max())


@pytest.mark.parametrize("T,w", [(24, 0.2), (5, 1.3)])
def test_forward_time_resolved_tally_parity(T, w):
    """The path-length (time-of-flight) resolved fluence against the oracle on the same streams:
    per bin relative L1 (a piece within FP32 rounding of a bin edge, or a path length summed in
    FP32 over hundreds of segments, may move a sliver to the neighbouring bin), and the bins sum
    to the plain run's a_0."""
    mua, mus = workloads.small_hetero(40, 52, 0.08, seed=14)
    src = _src32(dict(kind=mcr.LINE, x0=0.4, z0=0.0, x1=3.6, z1=0.0, dir_x=0.3, dir_z=1.0))
    dx, g = f32(0.08), f32(0.85)
    run = mcr.Run(K=0, n_packets=40_001, seed=19, time_bins=T, time_bin_mm=w)
    G = _gpu_forward(mua, mus, dx, g, src, run)
    O = oracle.forward(mua.astype(np.float64), mus.astype(np.float64), dx, g, src,
                       RunParams(K=0, n_packets=run.n_packets, seed=run.seed, time_bins=T, time_bin_mm=f32(w)))
    assert G.shape == O.coeff.shape == (T, 40, 52)
    tot = np.abs(O.coeff).sum()
    for b in range(T):
        assert np.abs(G[b] - O.coeff[b]).sum() <= 2e-3 * np.abs(O.coeff[b]).sum() + 1e-6 * tot, b
    a0 = _gpu_forward(mua, mus, dx, g, src, mcr.Run(K=0, n_packets=40_001, seed=19))[0]
    assert np.allclose(G.sum(axis=0), a0, rtol=2e-5, atol=1e-8 * a0.max())


def test_time_resolved_ballistic_closed_form_gpu():
    """mu_s = 0, pencil straight down the middle of column 4: pixel k is crossed over path lengths
    [k dx, (k+1) dx), so its fluence in bin b is the integral of e^{-mu_a L} over the overlap with
    [b w, (b+1) w) divided by dx^2 (FP32 transport: 1e-5)."""
    n, dx, mu, T, w = 12, 0.125, 0.75, 7, 0.15
    mua, mus = np.full((n, n), mu, np.float32), np.zeros((n, n), np.float32)
    G = _gpu_forward(mua, mus, dx, 0.3, dict(kind=mcr.PENCIL, x0=0.5625, z0=0.0, dir_x=0.0, dir_z=1.0),
                     mcr.Run(K=0, n_packets=1000, seed=2, time_bins=T, time_bin_mm=w))
    w = f32(w)
    want = np.zeros((T, n))
    for k in range(n):
        for b in range(T):
            lo, hi = max(k * dx, b * w), min((k + 1) * dx, (b + 1) * w if b < T - 1 else np.inf)
            if hi > lo:
                want[b, k] = (math.exp(-mu * lo) - math.exp(-mu * hi)) / mu / (dx * dx)
    assert np.allclose(G[:, :, 4], want, rtol=1e-5, atol=1e-6 * want.max())
    G[:, :, 4] = 0
    assert not G.any()


def test_time_resolved_tally_is_forward_only():
    mua, mus = workloads.small_hetero(8, 8, 0.1, seed=1)
    med = mcr.Medium(_dev(mua), _dev(mus), 0.1, 0.5)
    src = mcr.Source(kind=mcr.ISO_POINT, x0=0.4, z0=0.4)
    with pytest.raises(mcr.McrError):
        mcr.adjoint(med, torch.ones(8, 8, device="cuda"), mcr.Run(K=0, n_packets=100, time_bins=4, time_bin_mm=0.1))
    for bad in (dict(time_bins=4, time_bin_mm=0.0), dict(time_bins=4, time_bin_mm=0.1, sectors=3),
                dict(time_bins=2000, time_bin_mm=0.1)):
        with pytest.raises(mcr.McrError):
            mcr.forward(med, src, mcr.Run(K=0, n_packets=100, **bad))
    with pytest.raises(mcr.McrError):
        mcr.run_batch([mcr.Problem(med, 100, source=src)], mcr.Run(K=0, n_packets=0, time_bins=4, time_bin_mm=0.1))


def test_sector_tally_is_forward_only():
    mua, mus = workloads.small_hetero(8, 8, 0.1, seed=1)
    med = mcr.Medium(_dev(mua), _dev(mus), 0.1, 0.5)
    q = torch.ones(8, 8, device="cuda")
    with pytest.raises(mcr.McrError):
        mcr.adjoint(med, q, mcr.Run(K=0, n_packets=100, sectors=4))


def test_forward_oblique_pencil_K16_roulette():
    """Oblique pencil, strong absorption and a high threshold so that roulette is exercised.

    A packet whose weight lands within FP32 rounding of the threshold can take the other branch;
    1e6 packets (the packet count the 1e-4 bound is stated for) dilute such a packet below it."""
    mua, mus = workloads.small_hetero(33, 35, 0.1, seed=5)
    mua = mua * 8
    src = dict(kind=mcr.PENCIL, x0=1.3, z0=0.0, dir_x=0.5, dir_z=0.8, power=1.0)
    run = mcr.Run(K=16, n_packets=1_000_000, seed=2, w_threshold=0.05, roulette_p=0.25)
    G, O, st, _ = _forward_case(mua, mus, 0.1, 0.6, src, run, "pencil K16 roulette")
    assert O.stats["rr_kill"] > 100_000 and st["rr_kill"] > 100_000
    assert abs(st["rr_kill"] - O.stats["rr_kill"]) <= 1e-4 * O.stats["rr_kill"] + 5


def _adjoint_case(mua, mus, dx, g, q, run, label):
    dx, g = f32(dx), f32(g)
    med = mcr.Medium(_dev(mua), _dev(mus), dx, g)
    G, st = mcr.adjoint(med, _dev(q), run, stats=True)
    G = G.double().cpu().numpy()
    O = oracle.adjoint(mua.astype(np.float64), mus.astype(np.float64), dx, g, q, _orc_run(run))
    # absolute tally: the same packets with |W| (sampling uses |q*|, so the paths are identical)
    Oabs = oracle.adjoint(mua.astype(np.float64), mus.astype(np.float64), dx, g, np.abs(q), _orc_run(run),
                          with_variance=True)
    info = assert_parity(G, O.coeff, Oabs.coeff[0], np.sqrt(Oabs.a0_var), label=label)
    assert st["launched"] == run.n_packets
    assert abs(st["launched_w"] - O.stats["launched_w"]) == 0
    return G, O, st, info


def test_adjoint_signed_source_K16():
    mua, mus = workloads.small_hetero(40, 48, 0.08, seed=6)
    rng = np.random.default_rng(3)
    q = (rng.normal(size=mua.shape) * (rng.uniform(size=mua.shape) < 0.3)).astype(np.float32)
    run = mcr.Run(K=16, n_packets=50_003, seed=21, stream_id=1)
    _adjoint_case(mua, mus, 0.08, 0.8, q, run, "adjoint K16")


def test_adjoint_single_pixel_source_K8():
    mua, mus = workloads.small_hetero(24, 24, 0.1, seed=8)
    q = np.zeros(mua.shape, np.float32)
    q[5, 17] = -3.0
    run = mcr.Run(K=8, n_packets=40_000, seed=5)
    _adjoint_case(mua, mus, 0.1, 0.9, q, run, "adjoint point")


def test_gradient_h_eps_and_adjoint_source_parity():
    """mc_gradient / mc_h_eps / mc_adjoint_source vs the oracle functionals on the SAME seeded
    inputs (each kernel is fed numpy arrays, never another kernel's output)."""
    rng = np.random.default_rng(9)
    K, nz, nx, dx, g = 12, 37, 29, f32(0.05), f32(0.9)
    c = rng.normal(size=(2 * K + 1, nz, nx)).astype(np.float32)
    cs = rng.normal(size=(2 * K + 1, nz, nx)).astype(np.float32)
    c[0] = np.abs(c[0])
    mua = rng.uniform(0.01, 0.2, (nz, nx)).astype(np.float32)
    mus = rng.uniform(5, 20, (nz, nx)).astype(np.float32)
    Hm = rng.uniform(0, 0.5, (nz, nx)).astype(np.float32)
    med = mcr.Medium(_dev(mua), _dev(mus), dx, g)
    H, v, eps = mcr.h_eps(med, _dev(c), _dev(Hm))
    # expected values from the inputs alone: H is one FP32 product, computed here in numpy
    H32 = (mua * c[0]).astype(np.float32)
    assert np.array_equal(H.cpu().numpy(), H32)
    H64 = H32.astype(np.float64)
    assert abs(eps.item() - F.error_functional(Hm.astype(np.float64), H64, dx)) < 1e-12 * eps.item()
    v_ref = F.dL_dH_eps(Hm, H64, dx)
    assert np.allclose(v.cpu().numpy(), v_ref, rtol=1e-6, atol=0)
    vin = rng.normal(size=(nz, nx)).astype(np.float32)  # dL/dH input of the next two kernels
    q = mcr.adjoint_source(med, _dev(vin)).cpu().numpy()
    assert np.allclose(q, F.adjoint_source(mua, vin, dx), rtol=1e-6, atol=0)
    d_mua, d_mus = mcr.gradient(med, _dev(c), _dev(cs), _dev(vin))
    ra, rs = F.dL_dmu(c.astype(np.float64), cs.astype(np.float64), vin.astype(np.float64), dx, g)
    assert np.allclose(d_mua.cpu().numpy(), ra, rtol=1e-12, atol=1e-15 * np.abs(ra).max())
    assert np.allclose(d_mus.cpu().numpy(), rs, rtol=1e-12, atol=1e-15 * np.abs(rs).max())


def test_beer_lambert_closed_form_gpu():
    """mu_s = 0: one ray per packet; the GPU tally equals the Beer-Lambert closed form."""
    import test_oracle_pins as pins
    rng = np.random.default_rng(3)
    nz, nx, dx = 9, 11, f32(0.3)
    mua = rng.uniform(0.05, 1.5, (nz, nx)).astype(np.float32)
    mus = np.zeros((nz, nx), np.float32)
    th = math.radians(23.0)
    sx, sz = f32(math.sin(th)), f32(math.cos(th))
    x0 = f32(1.73)
    K = 5
    G = _gpu_forward(mua, mus, dx, 0.5, dict(kind=mcr.PENCIL, x0=x0, z0=0.0, dir_x=sx, dir_z=sz),
                     mcr.Run(K=K, n_packets=777))
    nrm = math.hypot(sx, sz)
    sx, sz = sx / nrm, sz / nrm
    exp = np.zeros_like(G)
    W = 1.0
    for iz, ix, l in pins._chords(x0, 0.0, sx, sz, nx, nz, dx):
        m = float(mua[iz, ix])
        exp[0, iz, ix] += W * (1 - math.exp(-m * l)) / m / (dx * dx)
        W *= math.exp(-m * l)
    th = math.atan2(sx, sz)
    for n in range(1, K + 1):
        exp[2 * n - 1] = exp[0] * math.cos(n * th)
        exp[2 * n] = exp[0] * math.sin(n * th)
    assert np.max(np.abs(G - exp)) <= 2e-5 * np.max(exp[0])


def test_energy_bookkeeping_gpu():
    """absorbed weight from the tally (sum mu_a a_0 A N_p) equals launched + roulette - escaped - killed."""
    mua, mus = workloads.small_hetero(40, 40, 0.1, seed=12)
    src = dict(kind=mcr.LINE, x0=0.0, z0=0.0, x1=4.0, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    run = mcr.Run(K=4, n_packets=500_000, seed=3, w_threshold=0.02, roulette_p=0.3, max_scatter=200)
    G, st = _gpu_forward(mua * 5, mus, 0.1, 0.8, src, run, stats=True)
    absorbed_tally = float(np.sum((mua * 5).astype(np.float64) * G[0])) * f32(0.1) ** 2 * run.n_packets
    assert st["rr_kill"] > 0 and st["scatter_limit"] > 0
    assert abs(absorbed_tally - st["absorbed_w"]) <= 1e-5 * st["launched_w"]


def test_bit_reproducible_and_packet_ranges_add_up():
    mua, mus = workloads.small_hetero(32, 32, 0.1, seed=13)
    src = dict(kind=mcr.LINE, x0=0.0, z0=0.0, x1=3.2, z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    a = _gpu_forward(mua, mus, 0.1, 0.9, src, mcr.Run(K=8, n_packets=100_000, seed=4))
    b = _gpu_forward(mua, mus, 0.1, 0.9, src, mcr.Run(K=8, n_packets=100_000, seed=4))
    assert np.array_equal(a, b)
    h1 = _gpu_forward(mua, mus, 0.1, 0.9, src, mcr.Run(K=8, n_packets=37_000, seed=4))
    h2 = _gpu_forward(mua, mus, 0.1, 0.9, src, mcr.Run(K=8, n_packets=63_000, seed=4, first_packet=37_000))
    comb = (h1 * 37_000 + h2 * 63_000) / 100_000
    assert np.allclose(comb, a, rtol=2e-6, atol=2e-7 * np.abs(a).max())


def test_edge_cases():
    dev = torch.device("cuda")
    # zero packets -> zeros; K = 0; a 1-pixel-wide grid
    mua, mus = np.full((7, 1), 0.1, np.float32), np.full((7, 1), 2.0, np.float32)
    src = dict(kind=mcr.PENCIL, x0=0.05, z0=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    z = _gpu_forward(mua, mus, 0.1, 0.5, src, mcr.Run(K=0, n_packets=0))
    assert z.shape == (1, 7, 1) and np.all(z == 0)
    G = _gpu_forward(mua, mus, 0.1, 0.5, src, mcr.Run(K=3, n_packets=20_000, seed=1))
    O = oracle.forward(mua.astype(np.float64), mus.astype(np.float64), f32(0.1), 0.5, _src32(src),
                       RunParams(K=3, n_packets=20_000, seed=1), with_variance=True)
    assert_parity(G, O.coeff, O.coeff[0], np.sqrt(O.a0_var), label="1-wide")
    # all-zero adjoint source -> zeros
    med = mcr.Medium(_dev(mua), _dev(mus), 0.1, 0.5)
    za = mcr.adjoint(med, torch.zeros((7, 1), device=dev), mcr.Run(K=2, n_packets=1000))
    assert torch.count_nonzero(za) == 0
    # a source outside the domain escapes at once
    Ge, st = _gpu_forward(mua, mus, 0.1, 0.5, dict(kind=mcr.PENCIL, x0=5.0, z0=0.0), mcr.Run(K=1, n_packets=64),
                          stats=True)
    assert st["escapes"] == 64 and np.all(Ge == 0)


def test_device_errors_are_reported():
    mua, mus = np.full((8, 8), 0.001, np.float32), np.full((8, 8), 50.0, np.float32)
    src = dict(kind=mcr.ISO_POINT, x0=0.4, z0=0.4, power=1.0)
    with pytest.raises(mcr.McrError) as e:
        _gpu_forward(mua, mus, 0.1, 0.0, src, mcr.Run(K=1, n_packets=100, max_events=3), stats=True)
    assert e.value.status == mcr.ERR_EVENT_LIMIT
    # without a stats request the event cap is latched on the device and reported by mc_check
    med_ok = mcr.Medium(_dev(mua), _dev(mus), 0.1, 0.0)
    mcr.forward(med_ok, mcr.Source(**src), mcr.Run(K=1, n_packets=100, max_events=3))
    with pytest.raises(mcr.McrError) as e:
        mcr.check()
    assert e.value.status == mcr.ERR_EVENT_LIMIT
    mcr.check()
    bad = mua.copy()
    bad[2, 3] = -1.0
    med = mcr.Medium(_dev(bad), _dev(mus), 0.1, 0.0)
    mcr.forward(med, mcr.Source(**src), mcr.Run(K=1, n_packets=100))
    with pytest.raises(mcr.McrError) as e:
        mcr.check()
    assert e.value.status == mcr.ERR_MEDIUM
    mcr.check()  # latched error is cleared once reported


def test_chunked_run_matches_closed_form():
    """More than 2^26 packets (two chunks with an FP64 flush): the mu_s = 0 tally is still exact."""
    nz, nx, dx = 4, 3, f32(0.2)
    mua = np.full((nz, nx), 0.5, np.float32)
    mus = np.zeros((nz, nx), np.float32)
    src = dict(kind=mcr.LINE, x0=0.0, z0=0.0, x1=f32(0.6), z1=0.0, dir_x=0.0, dir_z=1.0, power=1.0)
    n = (1 << 26) + 12345
    G = _gpu_forward(mua, mus, dx, 0.0, src, mcr.Run(K=1, n_packets=n, seed=3))
    col = np.array([(1 - math.exp(-0.5 * dx)) / 0.5 * math.exp(-0.5 * dx * k) for k in range(nz)]) / (dx * dx)
    frac = G[0] / col[:, None]  # each column receives ~1/3 of the packets
    assert np.allclose(frac.sum(axis=1), 1.0, rtol=1e-5)
    assert np.allclose(frac, 1 / 3, atol=5e-4)


@pytest.mark.parametrize("K,g", [(1, 0.0), (15, -0.9), (17, 0.99), (31, 0.5), (33, 0.3), (48, 0.8)])
def test_forward_every_deposit_split_and_extreme_anisotropy(K, g):
    """Every way the 2K+1 coefficients split between warp-wide chunks and the per-lane remainder
    (K = 17 and 33 leave three coefficients per lane, K = 15 and 31 fill partial chunks, K = 48
    one per lane), with isotropic, strongly backward and strongly forward scattering."""
    mua, mus = workloads.small_hetero(29, 37, 0.08, seed=40 + K)
    src = dict(kind=mcr.LINE, x0=0.0, z0=0.0, x1=2.96, z1=0.0, dir_x=0.2, dir_z=0.9, power=1.0)
    run = mcr.Run(K=K, n_packets=40_003, seed=K)
    _forward_case(mua, mus, 0.08, g, src, run, f"K{K} g{g}")


@pytest.mark.parametrize("K", [17, 33])
def test_adjoint_with_per_lane_remainder(K):
    mua, mus = workloads.small_hetero(26, 31, 0.1, seed=60 + K)
    q = np.random.default_rng(K).normal(size=(26, 31)).astype(np.float32)
    run = mcr.Run(K=K, n_packets=40_009, seed=K + 1, stream_id=1)
    _adjoint_case(mua, mus, 0.1, 0.7, q, run, f"adjoint K{K}")
