"""Batched persistent launches, CUDA-graph capture and a measuring autotuner.

Many illumination sources, wavelengths and grid sizes are independent forward (or adjoint)
problems.  ``mcr.run_batch`` runs up to 64 of them in ONE persistent transport launch, so the GPU
stays full until the last problem finishes instead of draining at the end of each.  This module
adds:

* ``BatchRunner`` -- holds a list of problems, runs them eagerly or replays them from a CUDA
  graph captured once (the packing, CDF, transport and finalize launches of the whole batch
  become one graph launch).  A graph replays the same packets (its seeds are baked in); build a
  new runner, or call ``recapture(seed)``, for a fresh ensemble.
* ``autotune`` -- times the candidate launch shapes (threads per block, resident blocks per SM,
  collision merge default/off/on, shared-memory tally for a small single problem) on the actual batch with CUDA events and keeps the fastest,
  cached per device, K and batch size.  Results do not depend on the shape (fixed-point
  tallies), only the time does.
"""
from __future__ import annotations

import json
import os
from dataclasses import replace

import torch

from . import mcr

DEFAULT_CANDIDATES = ((128, 0, 0), (128, 0, 1), (256, 0, 1), (64, 0, 2), (128, 4, 1), (256, 2, 0), (256, 0, 0, 2),
                      (128, 0, 2, 2))
_cache: dict = {}


def _key(problems, common: mcr.Run):
    name = torch.cuda.get_device_name()
    pixels = sum(p.medium.shape[0] * p.medium.shape[1] for p in problems)
    packets = sum(p.n_packets for p in problems)
    return f"{name}|K{common.K}|P{len(problems)}|px{pixels}|n{packets}"


def autotune(problems: list, common: mcr.Run, candidates=DEFAULT_CANDIDATES, reps: int = 2,
             cache_path: str | None = None) -> tuple:
    """Fastest (threads_per_block, blocks_per_sm, merge_collisions[, shared_tally]) for this
    batch, measured with CUDA events."""
    key = _key(problems, common)
    if key in _cache:
        return _cache[key]
    if cache_path and os.path.exists(cache_path):
        try:
            stored = json.load(open(cache_path))
            if key in stored:
                _cache[key] = tuple(stored[key]["launch"])
                return _cache[key]
        except (OSError, ValueError):
            pass
    stream = torch.cuda.current_stream()
    timings = {}
    mcr.run_batch(problems, common)  # warm-up, grows the workspace
    for cand in candidates:
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            try:
                mcr.run_batch(problems, common, launch=cand)
            except mcr.McrError:  # shape does not fit this K (shared memory): skip it
                break
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        if best < float("inf"):
            timings[cand] = best
    choice = min(timings, key=timings.get)
    _cache[key] = choice
    if cache_path:
        stored = {}
        if os.path.exists(cache_path):
            try:
                stored = json.load(open(cache_path))
            except (OSError, ValueError):
                stored = {}
        stored[key] = {"launch": list(choice), "ms": {"x".join(map(str, c)): ms for c, ms in timings.items()}}
        with open(cache_path, "w") as f:
            json.dump(stored, f, indent=1)
    return choice


class BatchRunner:
    """A fixed batch of problems, run eagerly or replayed from a captured CUDA graph."""

    def __init__(self, problems: list, common: mcr.Run, launch: tuple | None = None):
        self.problems = problems
        self.common = common
        self.launch = launch
        for p in problems:  # outputs are allocated once, so graph replays write in place
            p.c(common.K)
        self.graph = None

    @property
    def outputs(self):
        return [p.out for p in self.problems]

    def run(self, stats: bool = False):
        return mcr.run_batch(self.problems, self.common, launch=self.launch, stats=stats)

    def capture(self):
        """Capture the whole batch (pack, CDF, transport, finalize) into one CUDA graph."""
        self.run()  # sizes the library workspace outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                mcr.run_batch(self.problems, self.common, launch=self.launch, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.outputs

    def recapture(self, seed: int):
        """New seeds for every problem (a fresh ensemble) and a new graph."""
        for i, p in enumerate(self.problems):
            p.seed = seed
            p.stream_id = 2 * i
        self.graph = None
        return self.capture()
