"""Packet sharding of one run over several ranks (the multi-GPU form of the method), host logic on
CPU: two gloo ranks each tally their share of the packet range with fixed-point deposits (the
oracle's integer mode stands in for a GPU's mc_forward_raw), one int64 all-reduce sums them, and
the result equals the single-range run bit for bit.  Also: the shares partition the range, and a
share larger than one raw call is split into calls whose sums add up."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from oracle import RunParams
from paper_1608_05238_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUA = np.full((7, 6), 0.2)
MUS = np.full((7, 6), 5.0)
MUA[3:5, 2:4] = 1.0
SRC = dict(kind=oracle.LINE, x0=0.0, z0=0.0, x1=0.6, z1=0.0, dir_x=0.0, dir_z=1.0)
N, FIRST, K, Q = 1001, 77, 3, 28


def _sums(first, count):
    return torch.from_numpy(oracle.forward_sums(MUA, MUS, 0.1, 0.8, SRC, RunParams(
        K=K, n_packets=count, first_packet=first, seed=9, fixed_q=Q, n_threads=1)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="env://")
    share = shard.packet_range(rank, world, N, FIRST)
    total = shard.sharded_sums(_sums, N, FIRST)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, share, total.numpy()))


def test_two_ranks_sum_to_the_single_range_run_bit_for_bit():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, t0), (_, s1, t1) = res
    assert s0 == (FIRST, N // 2) and s1 == (FIRST + N // 2, N - N // 2)
    whole = _sums(FIRST, N).numpy()
    assert t0.dtype == np.int64 and np.array_equal(t0, whole) and np.array_equal(t1, whole)
    # the shards really differ (each rank ran its own packets), and a float sum would not be exact
    a, b = _sums(*s0).numpy(), _sums(*s1).numpy()
    assert not np.array_equal(a, whole) and np.array_equal(a + b, whole)


@pytest.mark.parametrize("world,n,first", [(1, 10, 0), (3, 10, 5), (4, 3, 0), (8, 1_000_003, 2 ** 40), (5, 0, 7)])
def test_packet_ranges_partition_the_run(world, n, first):
    shares = [shard.packet_range(r, world, n, first) for r in range(world)]
    assert shares[0][0] == first
    for (f0, c0), (f1, _) in zip(shares, shares[1:]):
        assert f0 + c0 == f1
    assert sum(c for _, c in shares) == n
    assert max(c for _, c in shares) - min(c for _, c in shares) <= 1


def test_share_split_into_raw_calls_adds_up(monkeypatch):
    """A share above the per-call limit runs as several calls into one tally (write, then add)."""
    monkeypatch.setattr(shard.mcr, "RAW_MAX_PACKETS", 64)
    calls = []

    def call(f, c, out, acc):
        calls.append((f, c, acc))
        t = _sums(f, c)
        if acc:
            out.add_(t)
        else:
            out.copy_(t)

    got = shard._raw_range(call, K, MUA.shape, "cpu", FIRST, 200)
    assert [c for _, c, _ in calls] == [64, 64, 64, 8] and [a for _, _, a in calls] == [False, True, True, True]
    assert torch.equal(got, _sums(FIRST, 200))
    calls.clear()
    empty = shard._raw_range(call, K, MUA.shape, "cpu", FIRST, 0)
    assert calls == [(FIRST, 0, False)] and not empty.any()


def test_sharded_sums_refuse_float_tallies():
    with pytest.raises(TypeError):
        shard.sharded_sums(lambda f, c: torch.zeros(3, dtype=torch.float64), 10)
