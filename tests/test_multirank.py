"""The benchmark's multi-rank host logic on CPU with the gloo backend (two ranks): independent
replicas (distinct packet seeds, no data exchange), the slowest rank's time, whole-job rate."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://")
    r, w, local = bench._dist()
    T = bench.max_over_ranks(1.0 + 0.5 * rank)  # rank 1 is the slow one
    seeds = [bench.replica_seed(r, k) for k in range(3)]
    value = bench.job_throughput(2e7, 3, w, T)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, T, seeds, value))


def test_two_gloo_ranks_take_the_slowest_time_and_draw_distinct_packets():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, T0, s0, v0), (r1, w1, l1, T1, s1, v1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert T0 == T1 == 1.5                      # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(2e7 * 3 * 2 / 1.5)
    assert not set(s0) & set(s1)                # replicas never share packet streams
    assert len(set(s0)) == 3


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_throughput(10, 2, 1, 4.0) == 5.0
