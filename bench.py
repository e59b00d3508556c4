"""Benchmark: one gradient evaluation of the forward + adjoint harmonic radiance MC per step.

Workload (``grad256``): 256 x 256 pixels of 0.05 mm, background mu_a 0.01 / mu_s 10 per mm,
g = 0.9, three random circular inclusions in the phantom that makes H^meas, collimated line
source on the top edge, K = 32 harmonics, 1e7 forward + 1e7 adjoint packets.  One step =
mc_forward -> mc_h_eps (H, eps, dL/dH) -> mc_adjoint_source -> mc_adjoint -> mc_gradient, all
CUDA kernels on one stream.  Metric: photons/s (forward + adjoint packets per second); the
gradient evaluations per second are the same number divided by 2e7.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (its own seeds) and rank 0
prints the whole-job rate (weak scaling, no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "photons/s fwd+adjoint harmonic MC; grad evals/s vs plain MC at stated error"
UNIT = "photons/s"
KERNELS_PER_STEP = 14  # pack, transport, finalize | h_eps x2 | adjoint source | pack, 4 cdf, transport, finalize | gradient


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--packets", type=int, default=10_000_000, help="packets per forward and per adjoint run")
    ap.add_argument("--cpu-sample", type=int, default=20_000, help="oracle packets (fwd and adj) for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload_config(w, n):
    return {"workload": f"grad256: {w.nx}x{w.nz} px of {w.dx} mm, 3 circular inclusions, g {w.g}, K={w.K}, "
                        f"line source on the top edge, {n:.0e} forward + {n:.0e} adjoint packets, gradient",
            "K": w.K, "pixels": [w.nz, w.nx], "dx_mm": w.dx, "packets_fwd": n, "packets_adj": n}


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------- oracle leg
def cpu_oracle_rate(w, Hmeas_np, n_sample: int, seed: int = 0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload (host cores)."""
    import oracle
    from oracle import RunParams
    from oracle import functionals as F
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    mua, mus = w.mua.astype(np.float64), w.mus.astype(np.float64)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    fw = oracle.forward(mua, mus, dx, g, w.sources[0], RunParams(K=w.K, n_packets=n_sample, seed=seed,
                                                                  n_threads=cores))
    H = F.absorbed_energy(mua, fw.coeff)
    v = F.dL_dH_eps(Hmeas_np, H, dx)
    q = F.adjoint_source(mua, v, dx).astype(np.float32)
    ad = oracle.adjoint(mua, mus, dx, g, q, RunParams(K=w.K, n_packets=n_sample, seed=seed + 1, stream_id=1,
                                                       n_threads=cores))
    F.dL_dmu(fw.coeff, ad.coeff, v, dx, g)
    dt = time.perf_counter() - t0
    return 2 * n_sample / dt, cores, dt


def _reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1608_05238_gb300 import workloads
    w = workloads.grad256(args.packets)
    # H^meas for the oracle leg: the phantom's absorbed energy from an oracle run (bounded sample)
    import oracle
    from oracle import RunParams
    from oracle import functionals as F
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    n = max(1000, args.cpu_sample // 10)
    hm = oracle.forward(w.mua_true.astype(np.float64), w.mus_true.astype(np.float64), dx, g, w.sources[0],
                        RunParams(K=0, n_packets=n, seed=1001))
    Hmeas = F.absorbed_energy(w.mua_true.astype(np.float64), hm.coeff)
    for k in range(args.warmup):
        cpu_oracle_rate(w, Hmeas, n, seed=10 * k)
    times = []
    for k in range(args.steps):
        rate, cores, dt = cpu_oracle_rate(w, Hmeas, n, seed=100 + 10 * k)
        times.append(dt)
    T = float(np.sum(times))
    value = 2 * n * args.steps / T
    sample = f"{n} forward + {n} adjoint packets per step of the grad256 workload (full 256x256 grid, K={w.K})"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _workload_config(w, args.packets),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------------- GPU leg
def _gpu(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1608_05238_gb300 import _build, mcr, workloads
    _build.build()
    w = workloads.grad256(args.packets)
    n = args.packets
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    stream = torch.cuda.current_stream()

    mua = torch.from_numpy(w.mua).to(dev)
    mus = torch.from_numpy(w.mus).to(dev)
    med = mcr.Medium(mua, mus, dx, g)
    src = mcr.Source(**w.sources[0])
    # H^meas: the phantom's absorbed energy from a separate 1e7-packet run (seed 1001), made once
    med_t = mcr.Medium(torch.from_numpy(w.mua_true).to(dev), torch.from_numpy(w.mus_true).to(dev), dx, g)
    Hmeas = mcr.h_eps(med_t, mcr.forward(med_t, src, mcr.Run(K=0, n_packets=n, seed=w.meta["hmeas_seed"])))
    coeff = torch.empty((2 * w.K + 1, w.nz, w.nx), dtype=torch.float32, device=dev)
    coeff_adj = torch.empty_like(coeff)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(k, m=med, hm=Hmeas):
        base = 1_000_003 * rank + 7919 * k
        mcr.forward(m, src, mcr.Run(K=w.K, n_packets=n, seed=base), out=coeff)
        H, v, eps = mcr.h_eps(m, coeff, hm)
        q = mcr.adjoint_source(m, v)
        mcr.adjoint(m, q, mcr.Run(K=w.K, n_packets=n, seed=base, stream_id=1), out=coeff_adj)
        return mcr.gradient(m, coeff, coeff_adj, v), eps

    for k in range(args.warmup):
        step(-1 - k)
    torch.cuda.synchronize()
    mcr.check()

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tr_ms, segs = [], []
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the timed events)
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
        ev[k][1].synchronize()
        for which in ("forward", "adjoint"):
            st, ms = mcr.last_run_info(which)
            tr_ms.append(ms)
            segs.append(st["segments"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    mcr.check()
    T = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([T], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        T = float(t.item())
        dist.barrier()
    value = 2 * n * args.steps * world / T

    # end to end through the public API: pinned host inputs -> device, result -> host, each step
    h_mua = torch.from_numpy(w.mua).pin_memory()
    h_mus = torch.from_numpy(w.mus).pin_memory()
    h_hm = Hmeas.cpu().pin_memory()
    d_mua, d_mus, d_hm = torch.empty_like(mua), torch.empty_like(mus), torch.empty_like(Hmeas)
    out_a = torch.empty((w.nz, w.nx), dtype=torch.float64).pin_memory()
    out_s = torch.empty_like(out_a)
    out_e = torch.empty((), dtype=torch.float64).pin_memory()
    h2d = 3 * 4 * w.nx * w.nz
    d2h = 2 * 8 * w.nx * w.nz + 8
    e2e_T = 0.0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_mua.copy_(h_mua, non_blocking=True)
        d_mus.copy_(h_mus, non_blocking=True)
        d_hm.copy_(h_hm, non_blocking=True)
        (ga, gs), eps = step(1000 + k, mcr.Medium(d_mua, d_mus, dx, g), d_hm)
        out_a.copy_(ga, non_blocking=True)
        out_s.copy_(gs, non_blocking=True)
        out_e.copy_(eps, non_blocking=True)
        torch.cuda.synchronize()
        e2e_T += time.perf_counter() - t0
    e2e_val = 2 * n * args.steps / e2e_T

    # roofline of the dominant kernel (the transport): algorithmic bytes = (2K+1) fixed-point
    # read-modify-writes of 8 B per pixel segment; achieved = bytes / event-timed kernel duration
    C = 2 * w.K + 1
    launches = len(tr_ms)
    avg_ms = float(np.mean(tr_ms))
    avg_segs = float(np.mean(segs))
    achieved_gbs = C * 8 * avg_segs / (avg_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                "traffic": None, "kernel": "k_transport", "launch_ms": avg_ms, "launches_timed": launches,
                "segments_per_launch": avg_segs, "bytes_per_segment": C * 8,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        hm_np = Hmeas.double().cpu().numpy()
        rate, cores, dt = cpu_oracle_rate(w, hm_np, args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} forward + {args.cpu_sample} adjoint packets of grad256 "
                         f"(full grid, K={w.K}), {dt:.1f} s"}

    if rank == 0:
        cfg = _workload_config(w, n)
        cfg.update({"l2": "flushed between timed steps (256 MB write)", "grad_evals_per_s": value / (2 * n),
                    "parallelism": f"replicas{world}" if world > 1 else "single"})
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient)", "data": "synthetic",
               "config": cfg, "clocks": clk,
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": KERNELS_PER_STEP * args.steps, "roofline": roofline, "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return _reference(args)
    return _gpu(args)


if __name__ == "__main__":
    sys.exit(main())
