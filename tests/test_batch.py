"""Batched persistent launch (mc_run_batch), CUDA-graph replay and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
from oracle import RunParams
from paper_1608_05238_gb300 import _build, batch, mcr, workloads
from parity_util import assert_parity, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    mcr.load()


def _medium(nz, nx, dx, g, seed):
    mua, mus = workloads.small_hetero(nz, nx, dx, seed=seed)
    return mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(g)), mua, mus


def _mixed_problems(K):
    """Forward and adjoint problems on uneven grids with different sources and packet counts."""
    probs, meta = [], []
    shapes = [(40, 56, 0.1), (33, 33, 0.05), (64, 24, 0.08), (17, 90, 0.12), (50, 50, 0.07), (26, 38, 0.09),
              (30, 44, 0.1)]
    for i, (nz, nx, dx) in enumerate(shapes):
        med, mua, mus = _medium(nz, nx, dx, 0.6 + 0.05 * i, seed=30 + i)
        n = 20_000 + 7_777 * i
        if i % 2 == 0:
            kinds = [mcr.Source(mcr.LINE, x0=0.0, z0=0.0, x1=f32(nx * dx), z1=0.0, dir_x=0.0, dir_z=1.0),
                     mcr.Source(mcr.ISO_POINT, x0=f32(0.37 * nx * dx), z0=f32(0.61 * nz * dx), power=2.0),
                     mcr.Source(mcr.PENCIL, x0=f32(0.5 * nx * dx), z0=0.0, dir_x=0.3, dir_z=0.9),
                     mcr.Source(mcr.ANGULAR_POINT, x0=f32(0.41 * nx * dx), z0=f32(0.45 * nz * dx),
                                ang_c=(0.0, 0.5), ang_s=(0.25,))]
            p = mcr.Problem(med, n, seed=5 + i, stream_id=2 * i, source=kinds[(i // 2) % 4])
            q = None
        else:
            q = np.random.default_rng(i).normal(size=(nz, nx)).astype(np.float32)
            q[np.random.default_rng(i + 9).uniform(size=q.shape) < 0.5] = 0
            p = mcr.Problem(med, n, seed=5 + i, stream_id=2 * i + 1, qstar=torch.from_numpy(q).cuda())
        probs.append(p)
        meta.append((mua, mus, q))  # the numpy inputs, for the oracle
    return probs, meta


def test_batch_equals_separate_calls_bit_for_bit():
    K = 16
    common = mcr.Run(K=K, n_packets=0)
    probs, _ = _mixed_problems(K)
    outs, st = mcr.run_batch(probs, common, stats=True)
    assert st["launched"] == sum(p.n_packets for p in probs)
    for p, o in zip(probs, outs):
        run = mcr.Run(K=K, n_packets=p.n_packets, seed=p.seed, stream_id=p.stream_id)
        ref = mcr.forward(p.medium, p.source, run) if p.source is not None else mcr.adjoint(p.medium, p.qstar, run)
        assert torch.equal(o, ref)


def test_batch_problem_matches_oracle():
    K = 16
    common = mcr.Run(K=K, n_packets=0)
    probs, meta = _mixed_problems(K)
    outs = mcr.run_batch(probs, common)
    for i in (0, 3):
        p, (mua, mus, qn) = probs[i], meta[i]
        rp = RunParams(K=K, n_packets=p.n_packets, seed=p.seed, stream_id=p.stream_id)
        args = (mua.astype(np.float64), mus.astype(np.float64), p.medium.dx, p.medium.g)
        if p.source is not None:
            O = oracle.forward(*args, p.source.as_dict(), rp, with_variance=True)
            A, sig = O.coeff[0], np.sqrt(O.a0_var)
        else:
            O = oracle.adjoint(*args, qn, rp)
            Oa = oracle.adjoint(*args, np.abs(qn), rp, with_variance=True)
            A, sig = Oa.coeff[0], np.sqrt(Oa.a0_var)
        assert_parity(outs[i].double().cpu().numpy(), O.coeff, A, sig, label=f"batch problem {i}")


def test_launch_shape_does_not_change_results_and_autotuner_picks_one():
    K = 8
    common = mcr.Run(K=K, n_packets=0)
    probs, _ = _mixed_problems(K)
    ref = [o.clone() for o in mcr.run_batch(probs, common)]
    for shape in ((64, 0), (256, 1, 1), (96, 3, 2), (128, 0, 1), (128, 0, 2)):
        outs = mcr.run_batch(probs, common, launch=shape)
        assert all(torch.equal(a, b) for a, b in zip(outs, ref))
    choice = batch.autotune(probs, common, reps=1)
    assert choice in batch.DEFAULT_CANDIDATES


@pytest.mark.parametrize("K", [8, 32, 64])
def test_collision_merge_is_bit_identical(K):
    """Depositing a surviving collision's segment together with the packet's next one changes
    only the number of L2 reductions, not the integer tally: also with roulette, the scatter cap
    and the event cap cutting packets off right at a collision."""
    med, _, _ = _medium(48, 40, 0.06, 0.8, seed=77)
    src = mcr.Source(mcr.LINE, x0=0.0, z0=0.0, x1=f32(40 * 0.06), z1=0.0, dir_x=0.0, dir_z=1.0)
    q = torch.from_numpy(np.random.default_rng(3).normal(size=(48, 40)).astype(np.float32)).cuda()
    for run in (mcr.Run(K=K, n_packets=0),
                mcr.Run(K=K, n_packets=0, w_threshold=0.6, roulette_p=0.5, max_scatter=40, max_events=25)):
        probs = [mcr.Problem(med, 30_000, seed=11, stream_id=0, source=src),
                 mcr.Problem(med, 30_000, seed=11, stream_id=1, qstar=q)]
        for pr in probs:
            outs = [mcr.run_batch([pr], run, launch=(128, 0, m))[0].clone() for m in (1, 2)]
            assert torch.equal(outs[0], outs[1])
        both = [[o.clone() for o in mcr.run_batch(probs, run, launch=(128, 0, m))] for m in (1, 2)]
        assert all(torch.equal(a, b) for a, b in zip(*both))
        # a packet ended by the event cap is latched on the device; mc_check reports and clears it
        try:
            mcr.check()
        except mcr.McrError as e:
            assert run.max_events == 25 and e.status == mcr.ERR_EVENT_LIMIT
        mcr.check()


def test_graph_replay_reproduces_eager_run():
    K = 16
    common = mcr.Run(K=K, n_packets=0)
    probs, _ = _mixed_problems(K)
    runner = batch.BatchRunner(probs, common)
    eager = [o.clone() for o in runner.run()]
    runner.capture()
    for o in runner.outputs:
        o.fill_(float("nan"))
    runner.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(runner.outputs, eager))
    runner.recapture(seed=77)
    runner.replay()
    torch.cuda.synchronize()
    assert not torch.equal(runner.outputs[0], eager[0])  # a new ensemble


def test_batch_limits():
    K = 4
    common = mcr.Run(K=K, n_packets=0)
    med, _, _ = _medium(8, 8, 0.1, 0.5, seed=1)
    src = mcr.Source(mcr.PENCIL, x0=0.4)
    with pytest.raises(ValueError):
        mcr.run_batch([mcr.Problem(med, 10, source=src)] * 65, common)
    with pytest.raises(mcr.McrError):
        mcr.run_batch([mcr.Problem(med, (1 << 26) + 1, source=src)], common)
    outs = mcr.run_batch([mcr.Problem(med, 0, source=src), mcr.Problem(med, 1000, source=src)], common)
    assert torch.count_nonzero(outs[0]) == 0 and torch.count_nonzero(outs[1]) > 0
    probs = [mcr.Problem(med, 100, seed=i, source=src) for i in range(64)]
    outs = mcr.run_batch(probs, common)
    assert all(torch.count_nonzero(o) > 0 for o in outs)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("K,n_small", [(8, 32), (16, 16)])
def test_shared_memory_tally_is_bit_identical(adjoint, K, n_small):
    """A per-block shared-memory copy of a small tally (32x32 at K = 8; 16x16 at K = 16, whose 33
    coefficients take the dense rows: 32 cooperative, coefficient 0 summed per lane) adds up to the
    same integer tally as the global one; a tally too large for shared memory falls back to the
    global one."""
    run = mcr.Run(K=K, n_packets=0, w_threshold=0.05, roulette_p=0.3)
    for n in (n_small, 80):
        med, _, _ = _medium(n, n, 0.25, 0.8, seed=91)
        if adjoint:
            q = torch.from_numpy(np.random.default_rng(5).normal(size=(n, n)).astype(np.float32)).cuda()
            prob = mcr.Problem(med, 300_000, seed=4, stream_id=1, qstar=q)
        else:
            src = mcr.Source(mcr.PENCIL, x0=f32(n * 0.25 / 2 + 0.1), z0=0.0, dir_x=0.0, dir_z=1.0)
            prob = mcr.Problem(med, 300_000, seed=4, stream_id=0, source=src)
        ref = mcr.run_batch([prob], run, launch=(128, 0, 1, 1))[0].clone()
        for shape in ((128, 0, 1, 2), (256, 0, 2, 2), (64, 0, 0, 2)):
            got = mcr.run_batch([prob], run, launch=shape)[0]
            assert torch.equal(got, ref), (n, shape)


def test_launch_order_is_bit_identical():
    """Packets processed in the order of their launch position (line sources by position along the
    line, volumetric sources by 32 x 32-pixel tile) give the same integer tallies as the launch
    index order, for single problems and for a mixed batch, with and without the collision merge."""
    K = 16
    probs, _ = _mixed_problems(K)
    common = mcr.Run(K=K, n_packets=0)
    for merge in (1, 2):
        ref = [o.clone() for o in mcr.run_batch(probs, common, launch=(128, 0, merge, 0, 1))]
        got = [o.clone() for o in mcr.run_batch(probs, common, launch=(128, 0, merge, 0, 2))]
        assert all(torch.equal(a, b) for a, b in zip(ref, got))
        for pr in probs[:3]:
            one = mcr.run_batch([pr], common, launch=(128, 0, merge, 0, 2))[0].clone()
            assert torch.equal(one, mcr.run_batch([pr], common, launch=(128, 0, merge, 0, 1))[0])


def test_large_tally_runs_ordered_by_default_and_matches_unordered():
    """A tally beyond 96 MB (768^2 pixels at K = 32: 377 MB) takes the launch order by default in
    mc_forward and mc_adjoint; the results equal the unordered batched launch bit for bit."""
    n, dx, K = 768, 0.02, 32
    mua, mus = workloads.inclusion_phantom(n, dx, 4, seed=3, margin=2.0)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(0.9))
    src = mcr.Source(**workloads.top_line_source(n, dx))
    run = mcr.Run(K=K, n_packets=100_000, seed=5)
    fwd = mcr.forward(med, src, run)
    ref = mcr.run_batch([mcr.Problem(med, 100_000, seed=5, source=src)], mcr.Run(K=K, n_packets=0),
                        launch=(0, 0, 0, 0, 1))[0]
    assert torch.equal(fwd, ref)
    q = torch.from_numpy(workloads.residual_source(n, dx, 7)).cuda()
    adj = mcr.adjoint(med, q, mcr.Run(K=K, n_packets=100_000, seed=6, stream_id=1))
    ref = mcr.run_batch([mcr.Problem(med, 100_000, seed=6, stream_id=1, qstar=q)], mcr.Run(K=K, n_packets=0),
                        launch=(0, 0, 0, 0, 1))[0]
    assert torch.equal(adj, ref)


@pytest.mark.parametrize("K", [8, 16, 32, 64])
def test_sorted_record_deposit_is_bit_identical(K):
    """The sorted-record deposit (records of every segment, counting-sorted by pixel, each pixel's
    run summed in registers) against the direct deposit, forward (line source) and adjoint: the
    integer tallies and the run counters are identical whether the records of a chunk fit the
    buffer, some chunks overflow it and run again directly, or every chunk does."""
    med, _, _ = _medium(72, 64, 0.06, 0.85, seed=91)
    src = mcr.Source(mcr.LINE, x0=0.0, z0=0.0, x1=f32(64 * 0.06), z1=0.0, dir_x=0.2, dir_z=1.0)
    q = torch.from_numpy(np.random.default_rng(4).normal(size=(72, 64)).astype(np.float32)).cuda()
    common = mcr.Run(K=K, n_packets=0)
    for pr in (mcr.Problem(med, 30_001, seed=12, source=src), mcr.Problem(med, 20_003, seed=13, stream_id=1, qstar=q)):
        ref, st_ref = mcr.run_batch([pr], common, launch=(128, 0, 0, 0, 0, 1, 0), stats=True)
        ref = ref[0].clone()
        for cap in (0, 60_000, 100):  # default buffer; chunks that sometimes overflow; always overflows
            got, st = mcr.run_batch([pr], common, launch=(128, 0, 0, 0, 0, 2, cap), stats=True)
            assert torch.equal(got[0], ref), cap
            for k in ("launched", "flights", "collisions", "segments", "escapes", "rr_kill", "rr_survive"):
                assert st[k] == st_ref[k], (cap, k)


def test_large_single_problem_takes_the_sorted_record_deposit_by_default():
    """Above 256 MB of tally (640^2 px at K = 64: 472 MB) mc_forward takes the sorted-record deposit;
    it equals the direct deposit of the batched call bit for bit."""
    n, dx, K = 640, 0.02, 64
    mua, mus = workloads.inclusion_phantom(n, dx, 4, seed=8, margin=2.0)
    med = mcr.Medium(torch.from_numpy(mua).cuda(), torch.from_numpy(mus).cuda(), f32(dx), f32(0.9))
    src = mcr.Source(**workloads.top_line_source(n, dx))
    fwd = mcr.forward(med, src, mcr.Run(K=K, n_packets=50_000, seed=3))
    ref = mcr.run_batch([mcr.Problem(med, 50_000, seed=3, source=src)], mcr.Run(K=K, n_packets=0),
                        launch=(0, 0, 0, 0, 0, 1, 0))[0]
    assert torch.equal(fwd, ref)
