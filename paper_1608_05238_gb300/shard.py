"""Packet sharding of one forward or adjoint run over several GPUs (one process per GPU).

The packets of a run are independent (Sec. 3: each packet's path depends only on its own random
numbers), so the packet range [first, first + N) of one problem splits into contiguous
sub-ranges, one per rank.  Each rank runs its sub-range with ``mc_forward_raw`` /
``mc_adjoint_raw`` into 64-bit fixed-point sums; one all-reduce (sum) of those int64 tallies
gives every rank the sums of the whole range -- integer addition is exact and order-free, so the
result is bit-identical to one GPU running all N packets -- and ``mc_finalize`` normalises them
with the total N.  This is the method's only exchange: the adjoint source is built from the
forward H of ALL packets, so the forward sums must be complete before the adjoint run starts.

The host logic here is written against a ``run_range(first, count) -> int64 tensor`` callable, so
the same code drives the CUDA library (the functions below) and, in the CPU tests, any other
producer of fixed-point sums.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable

import torch

from . import mcr


def world(group=None) -> tuple[int, int]:
    """(rank, world size) of ``group`` (the default group), or (0, 1) without torch.distributed."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def packet_range(rank: int, world_size: int, n: int, first: int = 0) -> tuple[int, int]:
    """Contiguous share (first_packet, count) of rank ``rank`` in [first, first + n): the shares of
    ranks 0 .. world_size-1 follow one another and cover the range exactly (sizes differ by <= 1)."""
    if not (0 <= rank < world_size) or n < 0:
        raise ValueError("bad rank / world size / packet count")
    lo = first + n * rank // world_size
    hi = first + n * (rank + 1) // world_size
    return lo, hi - lo


def sharded_sums(run_range: Callable[[int, int], torch.Tensor], n: int, first: int = 0, group=None) -> torch.Tensor:
    """Fixed-point sums of packets [first, first + n) over all ranks of ``group``: this rank's share
    from ``run_range``, then one int64 all-reduce (sum).  Every rank returns the same tensor."""
    rank, ws = world(group)
    lo, cnt = packet_range(rank, ws, n, first)
    tally = run_range(lo, cnt)
    if tally.dtype != torch.int64:
        raise TypeError("fixed-point sums must be int64 (an exact sum needs integers)")
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally


def _raw_range(call, K: int, shape, device, first: int, count: int) -> torch.Tensor:
    """Sums of packets [first, first + count) by calls of at most mcr.RAW_MAX_PACKETS packets,
    each after the first added into the same int64 tally."""
    out = torch.empty((2 * K + 1,) + tuple(shape), dtype=torch.int64, device=device)
    done = 0
    while True:  # the first call writes the tally (also for an empty range), later ones add
        c = min(count - done, mcr.RAW_MAX_PACKETS)
        call(first + done, c, out, done > 0)
        done += c
        if done >= count:
            return out


def forward(med: mcr.Medium, src: mcr.Source, run: mcr.Run, out=None, group=None) -> torch.Tensor:
    """mc_forward of ``run`` with its packets sharded over the ranks of ``group``; every rank gets
    the coefficients of all ``run.n_packets`` packets (``run.accumulate`` adds them into ``out``)."""
    def rr(first, count):
        return _raw_range(lambda f, c, o, acc: mcr.forward_raw(
            med, src, replace(run, first_packet=f, n_packets=c, accumulate=acc), out=o),
            run.K, med.shape, med.mua.device, first, count)
    tally = sharded_sums(rr, run.n_packets, run.first_packet, group)
    return mcr.finalize(med, run, tally, src=src, out=out)


def adjoint(med: mcr.Medium, qstar: torch.Tensor, run: mcr.Run, out=None, group=None) -> torch.Tensor:
    """mc_adjoint of ``run`` from ``qstar`` (identical on every rank) with its packets sharded."""
    def rr(first, count):
        return _raw_range(lambda f, c, o, acc: mcr.adjoint_raw(
            med, qstar, replace(run, first_packet=f, n_packets=c, accumulate=acc), out=o),
            run.K, med.shape, med.mua.device, first, count)
    tally = sharded_sums(rr, run.n_packets, run.first_packet, group)
    return mcr.finalize(med, run, tally, qstar=qstar, out=out)
