"""Benchmark: one gradient evaluation of the forward + adjoint harmonic radiance MC per step.

Workload (``grad256``): 256 x 256 pixels of 0.05 mm, background mu_a 0.01 / mu_s 10 per mm,
g = 0.9, three random circular inclusions in the phantom that makes H^meas, collimated line
source on the top edge, K = 32 harmonics, 1e7 forward + 1e7 adjoint packets.  One step is one
gradient evaluation through the autograd.Function: H = HFromMu(mu_a, mu_s) (mc_forward, H),
eps = EpsFromH(H, H^meas) (mc_eps), eps.backward() (mc_adjoint_source, mc_adjoint,
mc_gradient_f32), all libmcr kernels on one stream.  Metric: photons/s (forward + adjoint packets
per second); the gradient evaluations per second are the same number divided by 2e7.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) the ranks share the packets of ONE gradient evaluation: each rank runs its
contiguous range of every forward and adjoint run (1e7 + 1e7 packets per rank, so the work per GPU
stays fixed: weak scaling) into 64-bit fixed-point sums, one int64 all-reduce per run makes them
complete and bit-identical to a single GPU running all packets, and rank 0 prints the whole-job
rate.  ``--replicas`` runs independent replicas instead (own seeds, no data exchange).
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
# kernels of libmcr per step: forward (pack, transport, finalize, H) | eps (residual, reduction) |
# backward (adjoint source | pack, 4 CDF, transport, finalize | gradient)
KERNELS_PER_STEP = 15
# The L2's peak rate for reduction sectors on GB300 from ncu (lts__t_sectors_op_red.sum.peak_sustained
# = 188 sectors per cycle, lts__cycles_elapsed.avg.per_second = 2.017 GHz under load), times 32 B per
# sector: the ceiling of the transport's 64-bit tally reductions (profiles/k_transport_grad256_l2_reduction.md).
L2_RED_SECTORS_PER_CYCLE = 188
L2_CLOCK_HZ = 2.017e9
L2_RED_PEAK_GBS = L2_RED_SECTORS_PER_CYCLE * L2_CLOCK_HZ * 32 / 1e9
# DRAM bytes (read + write) per K = 32 transport launch of the grad256 gradient evaluation, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the benchmark's forward
# (40.36 MB) and adjoint (41.68 MB) launches at full size: the tally footprint, read once.
TRANSPORT_DRAM_BYTES = {"grad256": 41_017_344}
# DRAM bytes per pixel segment of the sorted-record deposit (transport in record mode, counting
# sort, deposit), from one ncu capture at 1024^2, K = 64 (1e6 packets, 1.327e9 segments: 126.3 GB;
# profiles/k_transport_large1024_records_dram.md), scaled to a launch by its segments.  Its
# algorithmic DRAM bytes: a 16-byte record written, read and rewritten by the sort, read by the deposit.
RECORD_DRAM_BYTES_PER_SEGMENT = 95.2
RECORD_ALG_BYTES_PER_SEGMENT = 64


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--packets", type=int, default=None,
                    help="packets per forward and per adjoint run (default 1e7 for grad256, 2e7 for large1024)")
    ap.add_argument("--cpu-sample", type=int, default=200_000, help="oracle packets (fwd and adj) for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent replicas instead of one packet-sharded gradient evaluation")
    ap.add_argument("--no-grad-error", action="store_true", help="skip the gradient-error measurement")
    ap.add_argument("--no-red-probe", action="store_true", help="skip the tally-reduction ceiling measurement")
    ap.add_argument("--plain-gd", action="store_true", help="invert256: no fluence preconditioning")
    ap.add_argument("--conv", default="128,128", help="conv: input,output channels of the timed 3x3 layer")
    ap.add_argument("--unknown", default=None, choices=["mua", "mus", "both"],
                    help="invert_rect: the reconstructed map (default mua); equal_error: mua, mus or both (default)")
    ap.add_argument("--iters", type=int, default=None, help="invert_rect, invert1024: iteration cap (default 20; 40 for mus)")
    ap.add_argument("--workload", default="grad256",
                    choices=["grad256", "large1024", "batch64", "denoise256", "conv", "invert256", "unet256", "invert_rect",
                             "sectors", "grad3d", "equal_error", "invert1024"],
                    help="grad256: the gradient evaluation (default); large1024: the same on 1024^2 px at "
                         "K = 64 with four edge sources; batch64: 64 forward problems in one graph-captured "
                         "batched launch; denoise256: the learned denoiser; conv: one large tensor-core "
                         "convolution (profiling case); invert256: mu_a reconstruction on the grad256 phantom; "
                         "unet256: U-Net training step and inference on synthetic maps (profiling case); invert_rect: "
                         "the Sec. 6 reconstructions on the rectangular-inclusion domain (--unknown mua|mus); sectors: "
                         "harmonic vs discrete-ordinates tally (Sec. 3.1); grad3d: the 3D gradient evaluation with "
                         "spherical-harmonic tallies (--n3 voxels a side, --l3 order); equal_error: the chosen form "
                         "(denoised low-count maps) against plain MC at equal reconstruction error (--unknown mua|mus); "
                         "invert1024: the 1024^2, K = 64 mu_a reconstruction, L-BFGS and gradient descent (--iters)")
    ap.add_argument("--pairs", type=int, default=1024, help="equal_error: training pairs per network")
    ap.add_argument("--train-steps", type=int, default=3000, help="equal_error: Adam steps per network")
    ap.add_argument("--nets", default=None,
                    help="equal_error: file of trained U-Net weights: loaded if it exists (no pairs made, no "
                         "training), else written after training")
    ap.add_argument("--methods", default="lbfgs_pre,gd_pre",
                    help="invert1024: comma list of lbfgs_pre, gd_pre (fluence-preconditioned), lbfgs, gd")
    ap.add_argument("--meas-packets", type=int, default=None,
                    help="invert1024: packets of the H^meas run (default 4x --packets, at least 1e8)")
    ap.add_argument("--chosen-packets", type=int, default=None,
                    help="equal_error: packets per MC run of the denoised route (default: the training inputs')")
    ap.add_argument("--train-low", type=int, default=100_000,
                    help="equal_error: packets of the training pairs' low-count inputs (targets: 1e7)")
    ap.add_argument("--n3", type=int, default=96, help="grad3d: voxels per side")
    ap.add_argument("--l3", type=int, default=4, help="grad3d: spherical-harmonic order L")
    args = ap.parse_args()
    if args.packets is None:
        args.packets = 20_000_000 if args.workload in ("large1024", "invert1024") else 10_000_000
    if args.unknown is None:
        args.unknown = "both" if args.workload == "equal_error" else "mua"
    if args.unknown == "both" and args.workload != "equal_error":
        ap.error("--unknown both applies to --workload equal_error only")
    if args.iters is None:
        args.iters = 40 if args.unknown == "mus" else 20
    return args


def _grad_workload(name, n):
    from paper_1608_05238_gb300 import workloads
    return workloads.large1024(n) if name == "large1024" else workloads.grad256(n)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank: int, k: int) -> int:
    """Seed of gradient evaluation k on rank ``rank``: each replica draws its own packets."""
    return 1_000_003 * rank + 7919 * k


def max_over_ranks(T: float, device=None) -> float:
    """The slowest rank's time (every rank calls this; any torch.distributed backend)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return T
    t = torch.tensor([T], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: float, steps: int, world: int, T: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_step * steps * world / T


def _workload_config(w, n):
    if w.name == "large1024":
        desc = (f"large1024: {w.nx}x{w.nz} px of {w.dx} mm, 8 circular inclusions, g {w.g}, K={w.K}, "
                f"4 line sources (one per edge, {n // 4:.1e} packets each) + {n:.0e} adjoint packets, gradient")
    else:
        desc = (f"grad256: {w.nx}x{w.nz} px of {w.dx} mm, 3 circular inclusions, g {w.g}, K={w.K}, "
                f"line source on the top edge, {n:.0e} forward + {n:.0e} adjoint packets, gradient")
    return {"workload": desc, "K": w.K, "pixels": [w.nz, w.nx], "dx_mm": w.dx, "packets_fwd": n, "packets_adj": n}


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
    """The FP64 oracle, as it stands, on a bounded sample of the same workload (host cores).
    The oracle keeps one FP64 tally per thread (1 GB at 1024^2, K = 64), so the large grid runs
    on 2 threads to bound host memory."""
    import oracle
    from oracle import RunParams
    from oracle import functionals as F
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    mua, mus = w.mua.astype(np.float64), w.mus.astype(np.float64)
    cores = os.cpu_count() or 1
    if w.nx * w.nz * (2 * w.K + 1) * 8 > (256 << 20):
        cores = min(cores, 2)
    t0 = time.perf_counter()
    per = max(1, n_sample // len(w.sources))
    fw = oracle.forward(mua, mus, dx, g, w.sources[0], RunParams(K=w.K, n_packets=per, seed=seed,
                                                                  n_threads=cores))
    fw_stats = dict(fw.stats)  # the first source's packets (per-photon work)
    for s in range(1, len(w.sources)):  # one illumination: the sources' fluences add
        fw.coeff += oracle.forward(mua, mus, dx, g, w.sources[s], RunParams(K=w.K, n_packets=per, seed=seed,
                                                                             stream_id=2 * s, n_threads=cores)).coeff
    H = F.absorbed_energy(mua, fw.coeff)
    v = F.dL_dH_eps(Hmeas_np, H, dx)
    q = F.adjoint_source(mua, v, dx).astype(np.float32)
    ad = oracle.adjoint(mua, mus, dx, g, q, RunParams(K=w.K, n_packets=n_sample, seed=seed + 1, stream_id=1,
                                                       n_threads=cores))
    F.dL_dmu(fw.coeff, ad.coeff, v, dx, g)
    dt = time.perf_counter() - t0
    fs, as_ = fw_stats, ad.stats
    work = {"forward": {"segments": fs["segments"] / fs["launched"], "collisions": fs["collisions"] / fs["launched"]},
            "adjoint": {"segments": as_["segments"] / as_["launched"], "collisions": as_["collisions"] / as_["launched"]}}
    return 2 * n_sample / dt, cores, dt, work


def oracle_hmeas(w, n):
    """H^meas for the oracle leg from an oracle run of the true medium (n packets per source, K = 0),
    so that no input of the oracle comes from the CUDA path."""
    import oracle
    from oracle import RunParams
    from oracle import functionals as F
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    mt, st = w.mua_true.astype(np.float64), w.mus_true.astype(np.float64)
    hm = oracle.forward(mt, st, dx, g, w.sources[0], RunParams(K=0, n_packets=n, seed=1001))
    for s in range(1, len(w.sources)):
        hm.coeff += oracle.forward(mt, st, dx, g, w.sources[s], RunParams(K=0, n_packets=n, seed=1001,
                                                                           stream_id=2 * s)).coeff
    return F.absorbed_energy(mt, hm.coeff)


def _reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    w = _grad_workload(args.workload, args.packets)
    n = max(1000, args.cpu_sample // (10 if w.name == "grad256" else 200))
    Hmeas = oracle_hmeas(w, n)
    for k in range(args.warmup):
        cpu_oracle_rate(w, Hmeas, n, seed=10 * k)
    times = []
    for k in range(args.steps):
        rate, cores, dt, _ = cpu_oracle_rate(w, Hmeas, n, seed=100 + 10 * k)
        times.append(dt)
    T = float(np.sum(times))
    value = 2 * n * args.steps / T
    sample = f"{n} forward + {n} adjoint packets per step of the {w.name} workload (full {w.nx}x{w.nz} grid, K={w.K})"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": _workload_config(w, args.packets),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------------- GPU leg
def l2_reduction_peak(rows, n_coeff, blocks=152 * 8, threads=256, iters=20000, reps=3, row_words=None):
    """Measured ceiling of the tally reductions (mc_reduction_probe): warps adding 1 to the first
    n_coeff 64-bit words of pseudo-random rows of a tally of this workload's shape, in the
    deposit's coalesced pattern, with no transport work.  Returns the best payload rate of
    ``reps`` event-timed runs (GB/s of 8-byte reductions) and checks the tally's total."""
    import torch
    from paper_1608_05238_gb300 import mcr
    if row_words is None:
        row_words = (n_coeff + 15) // 16 * 16 if n_coeff > 32 else (n_coeff + 3) // 4 * 4
    tally = torch.zeros(rows, row_words, dtype=torch.int64, device="cuda")
    mcr.reduction_probe(tally, n_coeff, 100, blocks, threads)  # warm-up
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mcr.reduction_probe(tally, n_coeff, iters, blocks, threads)
        b.record()
        b.synchronize()
        best = max(best, blocks * threads // 32 * iters * n_coeff * 8 / (a.elapsed_time(b) * 1e-3) / 1e9)
    warps = blocks * threads // 32
    assert int(tally.sum()) == warps * n_coeff * (100 + reps * iters), "reduction probe lost updates"
    return {"value": best, "unit": "GB/s", "how": f"mc_reduction_probe: {warps} warps x {iters} random rows of "
            f"{rows} x {row_words} int64, {n_coeff} coalesced 8-byte reductions per row, best of {reps}"}


def _gpu(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1608_05238_gb300 import _build, mcr
    from paper_1608_05238_gb300.autograd import EpsFromH, HFromMu, MCSpec, forward_coefficients
    _build.build()
    w = _grad_workload(args.workload, args.packets)
    n = args.packets
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    stream = torch.cuda.current_stream()

    mua = torch.from_numpy(w.mua).to(dev)
    mus = torch.from_numpy(w.mus).to(dev)
    srcs = [mcr.Source(**s) for s in w.sources]
    per_src = n // len(srcs)  # one illumination: the forward packets split over its sources
    # H^meas: the phantom's absorbed energy from a separate run (seed 1001), made once
    med_t = mcr.Medium(torch.from_numpy(w.mua_true).to(dev), torch.from_numpy(w.mus_true).to(dev), dx, g)
    Hmeas = mcr.h_eps(med_t, forward_coefficients(med_t, MCSpec(dx=dx, g=g, sources=srcs, K=0, n_packets=per_src,
                                                                 seed=w.meta["hmeas_seed"])))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    leaf_a = mua.clone().requires_grad_(True)
    leaf_s = mus.clone().requires_grad_(True)

    # N > 1: one problem whose packets are split over the ranks (same seeds on every rank, each
    # rank's share fixed at the 1-GPU packet count), or independent replicas (own seeds)
    sharded = world > 1 and not args.replicas
    share = world if sharded else 1

    def step(k, a=leaf_a, s=leaf_s, hm=Hmeas, scale=1):
        # one gradient evaluation through the autograd.Function: H(mu) -> eps -> backward
        base = replica_seed(0 if sharded else rank, k)
        spec = MCSpec(dx=dx, g=g, sources=srcs, K=w.K, n_packets=scale * per_src * share,
                      n_adjoint=scale * n * share, seed=base, adjoint_seed=base + 1, sharded=sharded)
        a.grad = None
        s.grad = None
        H = HFromMu.apply(a, s, spec)
        eps = EpsFromH.apply(H, hm, dx)
        eps.backward()
        return (a.grad, s.grad), eps

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
    work = {"forward": [0, 0, 0], "adjoint": [0, 0, 0]}  # launched, segments, collisions
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
            for i, key in enumerate(("launched", "segments", "collisions")):
                work[which][i] += st[key]
    torch.cuda.synchronize()
    clk = clocks.stop()
    mcr.check()
    T = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    n_fwd = per_src * len(srcs)
    value = job_throughput(n_fwd + n, args.steps, world, T)

    # end to end through the public API: pinned host inputs -> device, result -> host, each step
    h_mua = torch.from_numpy(w.mua).pin_memory()
    h_mus = torch.from_numpy(w.mus).pin_memory()
    h_hm = Hmeas.cpu().pin_memory()
    d_mua = torch.empty_like(mua).requires_grad_(True)
    d_mus = torch.empty_like(mus).requires_grad_(True)
    d_hm = torch.empty_like(Hmeas)
    out_a = torch.empty((w.nz, w.nx), dtype=torch.float32).pin_memory()
    out_s = torch.empty_like(out_a)
    out_e = torch.empty((), dtype=torch.float64).pin_memory()
    h2d = 3 * 4 * w.nx * w.nz
    d2h = 2 * 4 * w.nx * w.nz + 8
    e2e_T = 0.0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.no_grad():
            d_mua.copy_(h_mua, non_blocking=True)
            d_mus.copy_(h_mus, non_blocking=True)
            d_hm.copy_(h_hm, non_blocking=True)
        (ga, gs), eps = step(1000 + k, d_mua, d_mus, d_hm)
        out_a.copy_(ga, non_blocking=True)
        out_s.copy_(gs, non_blocking=True)
        out_e.copy_(eps, non_blocking=True)
        torch.cuda.synchronize()
        e2e_T += time.perf_counter() - t0
    e2e_val = job_throughput(n_fwd + n, args.steps, world, max_over_ranks(e2e_T, dev))

    # the error the rate is quoted at: relative L2 error of one gradient evaluation at this
    # packet count against one with 10x the packets (independent seeds); the reference's own
    # noise is 1/sqrt(10) of it, so the error proper is the measured one / sqrt(1.1)
    grad_err = None
    if rank == 0 and w.name == "grad256" and not args.no_grad_error:
        (ga, gs), _ = step(3000)
        ga, gs = ga.double().clone(), gs.double().clone()
        (ra, rs), _ = step(3001, scale=10)
        ra, rs = ra.double(), rs.double()
        ea = float((ga - ra).norm() / ra.norm()) / 1.1 ** 0.5
        es = float((gs - rs).norm() / rs.norm()) / 1.1 ** 0.5
        grad_err = {"d_eps_d_mua": ea, "d_eps_d_mus": es,
                    "how": "relative L2 error vs a 10x-packet evaluation, corrected for its noise"}

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
    # the tally reductions go to L2 (the grad256 tally is L2-resident): the bound is the L2's
    # reduction-sector rate; the HBM ratio is kept as a secondary figure
    row_words = (C + 15) // 16 * 16 if C > 32 else (C + 3) // 4 * 4
    # tallies beyond 256 MB take the sorted-record deposit: its roofline is HBM for the records
    in_hbm = w.nx * w.nz * row_words * 8 > 256 << 20
    if in_hbm:
        bound, peak = "hbm", hbm
        achieved_gbs = RECORD_ALG_BYTES_PER_SEGMENT * avg_segs / (avg_ms * 1e-3) / 1e9
    else:
        bound, peak = "l2_reduction", L2_RED_PEAK_GBS
    roofline = {"bound": bound, "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                "frac": achieved_gbs / peak,
                "traffic": (RECORD_DRAM_BYTES_PER_SEGMENT * avg_segs if in_hbm else TRANSPORT_DRAM_BYTES.get(w.name)),
                "kernel": "k_transport", "launch_ms": avg_ms, "launches_timed": launches,
                "segments_per_launch": avg_segs,
                "bytes_per_segment": RECORD_ALG_BYTES_PER_SEGMENT if in_hbm else C * 8,
                "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured): the tally lives in HBM" if in_hbm else
                                "ncu lts__t_sectors_op_red.sum.peak_sustained (188 sectors/cycle) x L2 clock "
                                "2.017 GHz x 32 B (of measured peak rate; profiles/k_transport_grad256_l2_reduction.md)"),
                "achieved_is": ("sorted-record deposit (transport + sort + deposit, event-timed): algorithmic DRAM "
                                "bytes 64 per segment (a 16-byte record written, read and rewritten by the sort, read "
                                "by the deposit); traffic = the measured 95.2 B per segment x segments.  The pipeline "
                                "is bound by its deposit kernel's instruction issue, far below HBM"
                                if in_hbm else
                                "algorithmic reduction payload 8 (2K+1) B per segment / event-timed launch")}
    if not in_hbm:
        roofline["hbm"] = {"peak": hbm, "frac": achieved_gbs / hbm,
                           "note": "payload rate over the measured HBM copy rate (MEASURED_PEAKS.json hbm_gbs); the "
                                   "payload goes to L2, DRAM sees `traffic` per launch"}
    if not args.no_red_probe:
        red = l2_reduction_peak(w.nx * w.nz, C)
        roofline["reduction_probe"] = dict(red, frac=achieved_gbs / red["value"],
                                           note="a measured rate of random-row reductions alone, not a ceiling")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        hm_np = oracle_hmeas(w, max(1000, args.cpu_sample // (10 if w.name == "grad256" else 200)))
        sample = args.cpu_sample if w.name == "grad256" else max(4, args.cpu_sample // 20)
        rate, cores, dt, owork = cpu_oracle_rate(w, hm_np, sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sample} forward + {sample} adjoint packets of {w.name} "
                         f"(full grid, K={w.K}), {dt:.1f} s", "work_per_photon": owork}

    if rank == 0:
        cfg = _workload_config(w, n)
        cfg["work_per_photon"] = {k: {"segments": v[1] / v[0], "collisions": v[2] / v[0]} for k, v in work.items()
                                  if v[0] > 0}
        cfg.update({"l2": "flushed between timed steps (256 MB write)", "grad_evals_per_s": value / ((n_fwd + n) * share),
                    "gradient_error_at_this_packet_count": grad_err,
                    "parallelism": (f"packet-sharded dp{world} (int64 all-reduce of the fixed-point sums)"
                                    if sharded else f"replicas{world}") if world > 1 else "single"})
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient)", "data": "synthetic",
               "config": cfg, "clocks": clk,
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               # sharded runs add one raw export per run and, for the adjoint, the source strength
               # (4 CDF kernels) in the finalisation
               "gpu_launches": (KERNELS_PER_STEP + 3 * (len(srcs) - 1) + (len(srcs) + 5 if sharded else 0))
               * args.steps, "roofline": roofline,
               "cpu_baseline": cpu}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _batch64(args):
    """64 forward problems (16 line sources x 4 wavelengths, 128^2/256^2/512^2 grids, K = 16,
    1e6 packets each) in one persistent batched launch, captured in a CUDA graph and replayed."""
    import torch
    from paper_1608_05238_gb300 import _build, batch, mcr, workloads
    _build.build()
    dev = torch.device("cuda", 0)
    n = min(args.packets, 1_000_000)
    specs = workloads.batch64(n)
    K = 16
    probs = []
    for s in specs:
        med = mcr.Medium(torch.from_numpy(s["mua"]).to(dev), torch.from_numpy(s["mus"]).to(dev),
                         float(np.float32(s["dx"])), float(np.float32(s["g"])))
        probs.append(mcr.Problem(med, s["n_packets"], seed=s["seed"], stream_id=s["stream_id"],
                                 source=mcr.Source(**s["source"])))
    common = mcr.Run(K=K, n_packets=0)
    launch = batch.autotune(probs, common, reps=1)
    runner = batch.BatchRunner(probs, common, launch=launch)
    _, st = runner.run(stats=True)
    runner.capture()
    for _ in range(args.warmup):
        runner.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    T = 0.0
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        runner.replay()
        b.record(stream)
        b.synchronize()
        T += a.elapsed_time(b) / 1e3
    clk = clocks.stop()
    mcr.check()
    total = n * len(probs)
    value = total * args.steps / T
    C = 2 * K + 1
    achieved = C * 8 * st["segments"] / (T / args.steps) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+i64", "data": "synthetic",
           "config": {"workload": f"batch64: 64 forward problems (16 line sources x 4 wavelengths) on 128^2/256^2/"
                                  f"512^2 grids of 12.8 mm, lognormal media, g 0.9, K={K}, {n:.0e} packets each, "
                                  f"one graph-captured batched launch", "launch": list(launch),
                      "tally_bytes": int(sum(p.medium.shape[0] * p.medium.shape[1] for p in probs) * 36 * 8),
                      "l2": "tallies (2.1 GB) exceed L2"},
           "clocks": clk, "gpu_launches": None,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "kernel": "k_transport (whole graph timed)",
                        "segments_per_launch": st["segments"], "bytes_per_segment": C * 8},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _unet_flops(net, B, H, W):
    """(algorithmic, executed) FLOPs of one U-Net forward pass on B images (2 per multiply-add);
    executed counts the channel padding the tensor-core tiles compute."""
    from paper_1608_05238_gb300.denoiser import UNet
    alg = exe = 0
    for name, lay in net.layers.items():
        P = B * (H >> UNet._level(name)) * (W >> UNet._level(name))
        alg += 2 * P * lay.cout * lay.taps * lay.cin
        exe += 2 * P * lay.n_pad * lay.taps * lay.cin_pad
    return alg, exe


def _denoise256(args):
    """The learned denoiser on 256x256 maps with K = 16 (33 channels): MC pair generation with the
    batched launch, training and inference with the tensor-core kernels, held-out error, and the
    throughput of one large tensor-core convolution against the measured BF16 peak."""
    import torch
    from paper_1608_05238_gb300 import _build, denoise_ops as ops, denoise_train as dt
    from paper_1608_05238_gb300.denoiser import UNet, sample_scale
    _build.build()
    K, n, dx = 16, 256, 0.05
    n_train, n_test, n_low, n_high = 128, 8, 100_000, 10_000_000
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    a, b = ev()
    a.record()
    x, t = dt.make_pairs(n_train + n_test, n=n, dx=dx, K=K, n_low=n_low, n_high=n_high)
    b.record()
    b.synchronize()
    gen_s = a.elapsed_time(b) / 1e3
    net = UNet(in_ch=2 * K + 1, seed=0)
    batch, steps = 8, max(50, args.steps * 300)
    dt.train(net, x[:n_train], t[:n_train], steps=3, batch=batch)  # warm-up
    a, b = ev()
    a.record()
    dt.train(net, x[:n_train], t[:n_train], steps=steps, batch=batch, lr=1e-3, seed=1)
    b.record()
    b.synchronize()
    train_s = a.elapsed_time(b) / 1e3
    ops.check()
    res = dt.evaluate(net, x[n_train:], t[n_train:])
    # equal-error comparison: plain MC at growing packet counts on the held-out phantoms
    curve = dt.plain_mc_error_curve(t[n_train:], [n_low, 2 * n_low, 4 * n_low, 8 * n_low], n=n, dx=dx, K=K,
                                    first=n_train)
    xb = x[:batch].contiguous()
    sc = sample_scale(xb)
    net.predict(xb, sc)
    a, b = ev()
    a.record()
    for _ in range(10):
        net.predict(xb, sc)
    b.record()
    b.synchronize()
    infer_s = a.elapsed_time(b) / 1e3 / 10
    alg, exe = _unet_flops(net, batch, n, n)
    ms_per_packet = np.polyfit([c[0] for c in curve], [c[3] for c in curve], 1)[0]
    ms_denoised = curve[0][3] + 1e3 * infer_s / batch  # n_low-packet MC map + its share of a batch inference
    equal = {}
    for which, key in ((1, "all_channels"), (2, "fluence_a0")):
        m_eq = dt.packets_at_error(curve, res["err_denoised" if which == 1 else "err_a0_denoised"], which)
        ms_plain = curve[0][3] + ms_per_packet * (m_eq - n_low)
        equal[key] = {"plain_mc_packets_at_denoised_error": m_eq, "plain_mc_ms_per_map": ms_plain,
                      "denoised_ms_per_map": ms_denoised, "speedup_at_equal_error": ms_plain / ms_denoised}
    # one large convolution (8 x 256 x 256 pixels, 128 -> 128 channels, 3x3) timed alone
    xc = torch.randn(8, 256, 256, 128, device="cuda").bfloat16()
    wc = (torch.randn(128, 9, 128, device="cuda") * 0.03).bfloat16()
    yc = torch.empty(8, 256, 256, 128, device="cuda", dtype=torch.bfloat16)
    for _ in range(3):
        ops.conv(xc, wc, 128, yc)
    a, b = ev()
    a.record()
    for _ in range(20):
        ops.conv(xc, wc, 128, yc)
    b.record()
    b.synchronize()
    conv_s = a.elapsed_time(b) / 1e3 / 20
    conv_tf = 2 * 8 * 256 * 256 * 128 * 9 * 128 / conv_s / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    out = {"metric": "denoised 256x256 K=16 maps/s (inference)", "value": batch / infer_s, "unit": "maps/s",
           "n_gpus": 1, "steps": steps, "warmup": 3, "ms_per_step": 1e3 * train_s / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
           "config": {"workload": f"denoise256: U-Net 32-256 ch on 33-channel 256^2 maps; {n_train} training + "
                                  f"{n_test} held-out MC pairs, inputs {n_low:.0e} packets, targets {n_high:.0e} "
                                  f"packets; batch {batch}",
                      "pair_generation_photons_per_s": (n_train + n_test) * (n_low + n_high) / gen_s,
                      "train_samples_per_s": steps * batch / train_s,
                      "train_tflops_executed": 3 * exe * steps / train_s / 1e12,
                      "infer_tflops_executed": exe / infer_s / 1e12,
                      "unet_forward_gflop_alg": alg / batch / 1e9, "unet_forward_gflop_executed": exe / batch / 1e9,
                      "heldout": res,
                      "plain_mc_curve": [{"packets": c[0], "err": c[1], "err_a0": c[2], "ms_per_map": c[3]}
                                         for c in curve],
                      "equal_error": equal},
           "roofline": {"bound": "tensor", "achieved": conv_tf, "peak": peak, "unit": "TFLOP/s", "frac": conv_tf / peak,
                        "traffic": None, "kernel": "k_conv_ws<2> (8x256x256, 128->128, 3x3, paired 256-pixel tiles)",
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)"},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _conv_only(args):
    """One 3x3 convolution and its weight gradient on 8 x 256 x 256 pixels (--conv CIN,COUT;
    default 128 -> 128 channels) on the tensor cores: the profiling case of the denoiser's
    convolution kernels."""
    import torch
    from paper_1608_05238_gb300 import _build, denoise_ops as ops
    from paper_1608_05238_gb300.denoise_ops import Act
    _build.build()
    cin, cout = (int(v) for v in args.conv.split(","))
    r64 = lambda c: (c + 63) // 64 * 64
    B, H, W = 8, 256, 256
    xc = torch.randn(B, H, W, r64(cin), device="cuda").bfloat16()
    wc = (torch.randn((cout + 15) // 16 * 16, 9, r64(cin), device="cuda") * 0.03).bfloat16()
    yc = torch.empty(B, H, W, r64(cout), device="cuda", dtype=torch.bfloat16)
    dw = torch.zeros(cout, 9, cin, device="cuda")
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for _ in range(args.warmup):
        ops.conv(xc, wc, cout, yc)
        ops.wgrad_nhwc(Act(yc, cout), Act(xc, cin), 9, dw)
    (a, b), (c, d) = ev(), ev()
    a.record()
    for _ in range(args.steps):
        ops.conv(xc, wc, cout, yc)
    b.record()
    c.record()
    for _ in range(args.steps):
        ops.wgrad_nhwc(Act(yc, cout), Act(xc, cin), 9, dw)
    d.record()
    d.synchronize()
    ops.check()
    s_conv, s_wg = a.elapsed_time(b) / 1e3 / args.steps, c.elapsed_time(d) / 1e3 / args.steps
    flop = 2 * B * H * W * cout * 9 * cin
    print(json.dumps({"metric": "conv TFLOP/s", "value": flop / s_conv / 1e12, "unit": "TFLOP/s",
                      "ms_per_step": 1e3 * s_conv, "config": {"workload": f"conv 8x256x256, {cin} -> {cout}, 3x3",
                                                              "wgrad_ms": 1e3 * s_wg,
                                                              "wgrad_tflops": flop / s_wg / 1e12}}), flush=True)
    return 0


def _unet256(args):
    """U-Net training step and inference on 8 synthetic 33-channel 256x256 maps (no MC pairs): the
    tensor-core convolutions, weight gradients and memory-bound layers of the denoiser alone
    (profiling case for its launch list)."""
    import torch
    from paper_1608_05238_gb300 import _build, denoise_ops as ops
    from paper_1608_05238_gb300.denoiser import UNet, sample_scale
    _build.build()
    B, C, H, W = 8, 33, 256, 256
    g = torch.Generator().manual_seed(0)
    x = (torch.rand(B, C, H, W, generator=g) + 0.5).cuda()
    t = (0.9 * x + 0.05).contiguous()
    net = UNet(in_ch=C, seed=0)
    sc = sample_scale(x)
    for _ in range(args.warmup):
        net.train_step(x, sc, t, 1e-4)
        net.predict(x, sc)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    (a, b), (c, d) = ev(), ev()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        net.train_step(x, sc, t, 1e-4)
    b.record()
    c.record()
    for _ in range(args.steps):
        net.predict(x, sc)
    d.record()
    d.synchronize()
    ops.check()
    train_ms, infer_ms = a.elapsed_time(b) / args.steps, c.elapsed_time(d) / args.steps
    alg, exe = _unet_flops(net, B, H, W)
    print(json.dumps({"metric": "U-Net training samples/s", "value": B / train_ms * 1e3, "unit": "samples/s",
                      "ms_per_step": train_ms, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
                      "config": {"workload": "unet256: U-Net 32-256 ch, batch 8 of 33-channel 256^2 maps",
                                 "infer_ms": infer_ms, "infer_maps_per_s": B / infer_ms * 1e3,
                                 "train_tflops_executed": 3 * exe / train_ms / 1e9,
                                 "infer_tflops_executed": exe / infer_ms / 1e9,
                                 "unet_forward_gflop_alg": alg / B / 1e9, "unet_forward_gflop_executed": exe / B / 1e9}}),
          flush=True)
    return 0


def _invert256(args):
    """mu_a reconstruction (Sec. 6.1: mu_s known) on the 256x256 inclusion phantom from a
    homogeneous start: (fluence-preconditioned, unless --plain-gd) gradient descent with the
    backtracking line search of inversion.py, one
    forward + one adjoint run per iteration plus the line search's forward runs, K = 10 (the
    paper's harmonic count for its inversions).  Reports the mean relative mu_a error after each
    accepted step and the wall time to reach it."""
    import torch
    from paper_1608_05238_gb300 import _build, mcr, workloads
    from paper_1608_05238_gb300.autograd import MCSpec, forward_coefficients
    from paper_1608_05238_gb300.inversion import invert, mean_relative_error
    _build.build()
    n_pk = args.packets
    w = workloads.grad256(n_pk)
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    dev = torch.device("cuda")
    mua_t = torch.from_numpy(w.mua_true).to(dev)
    mus_t = torch.from_numpy(w.mus_true).to(dev)
    srcs = [mcr.Source(**s) for s in w.sources]
    med_t = mcr.Medium(mua_t, mus_t, dx, g)
    Hmeas = mcr.h_eps(med_t, forward_coefficients(med_t, MCSpec(dx=dx, g=g, sources=srcs, K=0, n_packets=10 * n_pk,
                                                                 seed=w.meta["hmeas_seed"])))
    spec = MCSpec(dx=dx, g=g, sources=srcs, K=10, n_packets=n_pk)
    mua0 = torch.from_numpy(w.mua).to(dev)
    invert(mua0, mus_t, Hmeas, replace_spec(spec, n_packets=max(1000, n_pk // 100)), iters=1)  # warm-up
    torch.cuda.synchronize()
    iters = max(args.steps, 1) * 4
    t0 = time.perf_counter()
    res = invert(mua0, mus_t, Hmeas, spec, unknowns=("mua",), iters=iters, tol=1e-9, mua_true=mua_t,
                 precondition=not args.plain_gd)
    torch.cuda.synchronize()
    T = time.perf_counter() - t0
    e0 = mean_relative_error(mua0, mua_t)
    hist = [{"it": h.it, "eps": h.eps, "rel_err_mua": h.rel_err_mua, "seconds": h.seconds, "trials": h.trials}
            for h in res.history]
    runs = sum(2 + h.trials for h in res.history)
    out = {"metric": "mu_a reconstruction: mean relative error after the timed iterations", "value":
           res.history[-1].rel_err_mua if res.history else e0, "unit": "relative error", "n_gpus": 1,
           "steps": len(res.history), "warmup": 1, "ms_per_step": 1e3 * T / max(1, len(res.history)),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient)",
           "data": "synthetic",
           "config": {"workload": f"invert256: grad256 phantom (256x256 px of {w.dx} mm, 3 inclusions, g {w.g}), "
                                  f"mu_s known, homogeneous mu_a start, K=10, {n_pk:.0e} packets per MC run, "
                                  + ("plain gradient descent" if args.plain_gd else "fluence-preconditioned descent"),
                      "initial_rel_err_mua": e0, "seconds": T, "mc_runs": runs,
                      "photons_per_s": runs * n_pk / T, "history": hist},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _equal_error(args):
    """The chosen form against plain MC at equal reconstruction error (the paper's Sec. 6 metric,
    the mean relative error of the reconstructed map).  Both routes run the same reconstruction
    (inversion.invert: mu_a by fluence-preconditioned descent, or mu_s by backtracking under
    Eq. 30) on a held-out 256^2 inclusion phantom with K = 16 and the gradient from the autograd
    Function.  Plain: full MC maps at several packet counts per run.  Chosen: low-count maps
    (--chosen-packets per run, default the training inputs' --train-low, 1e5) through the U-Nets (forward and
    adjoint, trained here on MC pairs made by the batched launch, or loaded with --nets), judged
    once per kind by an MC run of 10x the packets (denoised.Denoiser).  The plain curve of error against
    packets per run, interpolated in log-log, gives the packet count -- and, from the measured time
    per iteration against packets, the time -- at which plain MC reaches the chosen form's error."""
    import torch
    from paper_1608_05238_gb300 import _build, denoise_train as dt, mcr, workloads
    from paper_1608_05238_gb300.autograd import MCSpec, forward_coefficients
    from paper_1608_05238_gb300.denoised import Denoiser
    from paper_1608_05238_gb300.denoiser import UNet
    from paper_1608_05238_gb300.inversion import invert, mean_relative_error
    _build.build()
    K, n, dx, g = 16, 256, 0.05, 0.9
    n_low, n_high, n_pairs, n_test = args.train_low, 10_000_000, args.pairs, 16
    dev = torch.device("cuda")
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    nets = {}
    if args.nets and os.path.exists(args.nets):
        saved = torch.load(args.nets)
        for kind in ("forward", "adjoint"):
            net = UNet(in_ch=2 * K + 1, seed=0)
            net.set_state(saved[kind]["state"])
            nets[kind] = (net, saved[kind]["heldout"])
        gen_s, train_s, n_pairs = saved["pair_generation_s"], saved["training_s"], saved["pairs"]
        n_low = saved.get("n_low", n_low)  # the inputs the saved networks were trained on
    else:
        t0 = time.perf_counter()
        xf, tf = dt.make_pairs(n_pairs + n_test, n=n, dx=dx, K=K, n_low=n_low, n_high=n_high, vary=True)
        xa, ta = dt.make_adjoint_pairs(n_pairs + n_test, n=n, dx=dx, K=K, n_low=n_low, n_high=n_high)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        for kind, (x, t) in (("forward", (xf, tf)), ("adjoint", (xa, ta))):
            net = UNet(in_ch=2 * K + 1, seed=1 if kind == "forward" else 2)
            dt.train(net, x[:n_pairs], t[:n_pairs], steps=args.train_steps, batch=8, lr=1e-3, seed=3)
            nets[kind] = (net, dt.evaluate(net, x[n_pairs:], t[n_pairs:]))
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del xf, tf, xa, ta
        torch.cuda.empty_cache()
        if args.nets:
            torch.save({"pairs": n_pairs, "n_low": n_low, "pair_generation_s": gen_s, "training_s": train_s,
                        **{k: {"state": v[0].state(), "heldout": v[1]} for k, v in nets.items()}}, args.nets)

    # the reconstructions: held-out phantom, homogeneous start in the unknown map
    dx32, g32 = float(np.float32(dx)), float(np.float32(g))
    mua_t_np, mus_t_np = workloads.inclusion_phantom(n, dx, 3, seed=30_001, mus_range=(5.0, 15.0))
    mua_t, mus_t = torch.from_numpy(mua_t_np).to(dev), torch.from_numpy(mus_t_np).to(dev)
    src = [mcr.Source(**workloads.top_line_source(n, dx))]
    med_t = mcr.Medium(mua_t, mus_t, dx32, g32)
    Hmeas = mcr.h_eps(med_t, forward_coefficients(med_t, MCSpec(dx=dx32, g=g32, sources=src, K=0,
                                                                 n_packets=100_000_000, seed=777)))
    unknowns = ("mua", "mus") if args.unknown == "both" else (args.unknown,)
    results = {}
    for unknown in unknowns:
        iters = args.iters if args.unknown != "both" else (20 if unknown == "mua" else 40)
        mua0 = torch.full_like(mua_t, 0.01) if unknown == "mua" else mua_t.clone()
        mus0 = torch.full_like(mus_t, 10.0) if unknown == "mus" else mus_t.clone()
        kw = dict(unknowns=(unknown,), iters=iters, tol=1e-12, mua_true=mua_t, mus_true=mus_t)
        kw.update(precondition=True) if unknown == "mua" else kw.update(armijo=0.2, shrink=0.5)
        true = mua_t if unknown == "mua" else mus_t
        start = mua0 if unknown == "mua" else mus0
        # mu_s: at these packet counts noise dominates the domain-wide error (the paper too reports
        # a partial mu_s reconstruction), so the comparison is made on the error over the
        # inclusions, where the mu_s contrast is; the domain-wide error is reported beside it
        incl = (mus_t != 10.0) if unknown == "mus" else None
        region_err = (lambda est: float(((est[incl] - mus_t[incl]).abs() / mus_t[incl]).mean().double())) \
            if unknown == "mus" else None
        if unknown == "mus":
            kw.update(monitor=lambda a, s_: {"rel_err_mus_inclusions": region_err(s_)})

        def route(n_pk, denoiser=None):
            spec = MCSpec(dx=dx32, g=g32, sources=src, K=K, n_packets=n_pk, denoiser=denoiser)
            torch.cuda.synchronize()
            a = time.perf_counter()
            res = invert(mua0, mus0, Hmeas, spec, seed0=11, **kw)
            torch.cuda.synchronize()
            T = time.perf_counter() - a
            if unknown == "mua":
                errs = [h.rel_err_mua for h in res.history]
                e_start = mean_relative_error(start, true)
            else:
                errs = [h.extra["rel_err_mus_inclusions"] for h in res.history]
                e_start = region_err(start)
            tail = errs[-4:] if errs else [e_start]
            evals = len(res.history) + sum(h.trials for h in res.history)  # gradients + line-search forwards
            out = {"packets_per_run": n_pk, "final_err": float(np.mean(tail)), "errors": errs, "seconds": T,
                   "iterations": len(res.history), "mc_evaluations": evals,
                   "grad_evals_per_s": len(res.history) / T if T > 0 else None}
            if unknown == "mus":
                out["domain_errors"] = [h.rel_err_mus for h in res.history]
            return out

        route(20_000)  # warm-up (workspaces, kernels)
        plain = [route(int(m)) for m in (1e5, 2e5, 4e5, 1e6, 2e6, 4e6)]
        n_run = args.chosen_packets or n_low  # the denoised route's packets per run
        dn = Denoiser(nets["forward"][0], nets["adjoint"][0], n_full=n_high, n_judge=10 * n_run, judge_every=0,
                      max_rel_err=0.6)
        # warm-up of everything the chosen route runs first (U-Net kernels, the judge's norms), as
        # route(20_000) is for the plain route: a throw-away denoiser with a cheap judge and fallback
        route(20_000, Denoiser(nets["forward"][0], nets["adjoint"][0], n_full=20_000, n_judge=20_000, judge_every=0,
                               max_rel_err=0.6))
        chosen = route(n_run, dn)
        chosen["judge"] = dn.history
        chosen["fallback"] = dn.fallback
        # plain MC at the chosen form's error: log-log fit of the plain error against packets per
        # run, and of its time against packets
        lm = np.log([p["packets_per_run"] for p in plain])
        le = np.log([p["final_err"] for p in plain])
        lt = np.log([p["seconds"] for p in plain])
        se, ie = np.polyfit(lm, le, 1)
        st, it_ = np.polyfit(lm, lt, 1)
        # no equal-error point when the chosen route took no step (its error is the start's)
        moved = chosen["iterations"] > 0
        m_eq = float(np.exp((np.log(chosen["final_err"]) - ie) / se)) if (se < 0 and moved) else None
        t_eq = float(np.exp(it_ + st * np.log(m_eq))) if m_eq else None
        results[unknown] = {"error_measure": ("mean relative mu_a error over the domain" if unknown == "mua" else
                                              "mean relative mu_s error over the inclusions"),
                            "initial_err": (mean_relative_error(start, true) if unknown == "mua" else
                                            region_err(start)),
                            "iterations": iters, "plain": plain,
                            "chosen": chosen, "plain_packets_per_run_at_chosen_error": m_eq,
                            "plain_seconds_at_chosen_error": t_eq, "plain_error_vs_packets_loglog_slope": float(se),
                            "speedup_at_equal_error": (t_eq / chosen["seconds"]) if t_eq else None,
                            "chosen_grad_evals_per_s": chosen["grad_evals_per_s"]}
    head = unknowns[0]
    value = results[head]["speedup_at_equal_error"]
    first = results[head]
    out = {"metric": "time to equal mean relative reconstruction error: plain MC / (batched + autograd + denoised)",
           "value": value, "unit": f"speedup at equal {head} error (the other maps: config.results)", "n_gpus": 1,
           "steps": first["iterations"], "warmup": 1,
           "ms_per_step": 1e3 * first["chosen"]["seconds"] / max(1, first["chosen"]["iterations"]),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+i64 (FP64 gradient), bf16 U-Net", "data": "synthetic",
           "config": {"workload": f"equal_error: {'/'.join(unknowns)} reconstruction, 256x256 px of {dx} mm, held-out "
                                  f"3-inclusion phantom (seed 30001), top line source, K={K}; U-Nets trained on "
                                  f"{n_pairs} forward + {n_pairs} adjoint MC pairs ({n_low:.0e} -> {n_high:.0e} packets); "
                                  f"denoised route at {args.chosen_packets or n_low:.0e} packets per run",
                      "pair_generation_s": gen_s, "training_s": train_s, "train_steps": args.train_steps,
                      "heldout_map_errors": {k: v[1] for k, v in nets.items()}, "results": results},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _invert1024(args):
    """The 1024^2 configuration's reconstruction: mu_a of the large1024 phantom (1024^2 px of 0.02
    mm, 8 inclusions, g 0.9, four edge line sources, K = 64, mu_s known), H^meas from --meas-packets
    packets of the true medium, started from the homogeneous background, by each of --methods for
    --iters iterations with --packets per MC run (split over the four sources for the forward runs):
    L-BFGS (the plan's optimiser) and gradient descent with the Hager-Zhang line search (the
    paper's, Sec. 6.1), each plain or with the fluence preconditioner (``_pre``: the diagonal
    1 / (dx^2 Phi^2) as L-BFGS's initial inverse Hessian, or as the descent's step scaling).  All use
    the gradient of the autograd Function (forward harmonics recomputed at K = 64) and the line
    searches' FP64 inner products on the GPU (mc_dot); the tallies take the sorted-record deposit
    (1.2 GB each).  Reports the mean relative mu_a error and eps per iteration and the time per
    iteration of each method; the headline is the first method's seconds per iteration."""
    import torch
    from paper_1608_05238_gb300 import _build, mcr, workloads
    from paper_1608_05238_gb300.autograd import MCSpec, forward_coefficients
    from paper_1608_05238_gb300.inversion import invert, mean_relative_error
    _build.build()
    methods = [m.strip() for m in args.methods.split(",") if m.strip()]
    for m in methods:
        if m not in ("lbfgs_pre", "gd_pre", "lbfgs", "gd"):
            raise SystemExit(f"unknown method {m!r}")
    w = workloads.large1024(args.packets)
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    dev = torch.device("cuda")
    mua_t, mus_t = torch.from_numpy(w.mua_true).to(dev), torch.from_numpy(w.mus_true).to(dev)
    srcs = [mcr.Source(**s) for s in w.sources]
    med_t = mcr.Medium(mua_t, mus_t, dx, g)
    n_meas = args.meas_packets or max(100_000_000, 4 * args.packets)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hmeas = mcr.h_eps(med_t, forward_coefficients(med_t, MCSpec(dx=dx, g=g, sources=srcs, K=0,
                                                                 n_packets=n_meas // len(srcs), seed=1001)))
    torch.cuda.synchronize()
    t_meas = time.perf_counter() - t0
    spec = MCSpec(dx=dx, g=g, sources=srcs, K=w.K, n_packets=args.packets // len(srcs), n_adjoint=args.packets)
    mua0 = torch.from_numpy(w.mua).to(dev)  # the homogeneous background
    e0 = mean_relative_error(mua0, mua_t)
    results = {}
    for method in methods:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = invert(mua0, mus_t, Hmeas, spec, unknowns=("mua",), iters=args.iters, tol=1e-12,
                     line_search="hager_zhang", method=method.replace("_pre", ""),
                     precondition=method.endswith("_pre"), mua_true=mua_t, seed0=17)
        torch.cuda.synchronize()
        T = time.perf_counter() - t0
        hist = [{"it": h.it, "eps": h.eps, "rel_err_mua": h.rel_err_mua, "seconds": h.seconds, "trials": h.trials}
                for h in res.history]
        evals = len(res.history) + sum(h.trials for h in res.history)
        results[method] = {"seconds": T, "iterations": len(res.history), "gradient_evaluations": evals,
                           "seconds_per_iteration": T / max(1, len(res.history)),
                           "final_rel_err_mua": res.history[-1].rel_err_mua if res.history else e0,
                           "history": hist}
    head = results[methods[0]]
    out = {"metric": f"1024^2 K=64 mu_a reconstruction: seconds per iteration ({methods[0]})", "value":
           head["seconds_per_iteration"], "unit": "s/iteration", "n_gpus": 1, "steps": head["iterations"],
           "warmup": 0, "ms_per_step": 1e3 * head["seconds_per_iteration"], "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient and inner products)",
           "data": "synthetic",
           "config": {"workload": f"invert1024: large1024 phantom (1024x1024 px of {w.dx} mm, 8 inclusions, g "
                                  f"{w.g}), mu_s known, homogeneous mu_a start, K={w.K}, {args.packets:.0e} "
                                  f"packets per forward (4 edge sources) and per adjoint run, H^meas from "
                                  f"{n_meas:.0e} ({t_meas:.1f} s)",
                      "initial_rel_err_mua": e0, "results": results},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _sectors(args):
    """Sec. 3.1's trade-off, measured: the forward transport of the 256^2 workload with the harmonic
    tally at K = 8, 16, 32 against the discrete-ordinates tally at M = 16, 32, 64 sectors -- tally
    words per pixel, transport rate, and the relative spread over seeds of one angular channel
    against that of the fluence at the same packet count."""
    import torch
    from paper_1608_05238_gb300 import _build, mcr, workloads
    _build.build()
    w = workloads.grad256(args.packets)
    dx, g = float(np.float32(w.dx)), float(np.float32(w.g))
    med = mcr.Medium(torch.from_numpy(w.mua).cuda(), torch.from_numpy(w.mus).cuda(), dx, g)
    src = mcr.Source(**w.sources[0])
    rows = []
    pix = (64, 128)  # 3.2 mm under the middle of the source line
    for label, K, M in [("harmonics", 8, 0), ("harmonics", 16, 0), ("harmonics", 32, 0), ("sectors", 0, 16),
                        ("sectors", 0, 32), ("sectors", 0, 64)]:
        mcr.forward(med, src, mcr.Run(K=K, n_packets=args.packets // 10, seed=1, sectors=M))  # warm-up
        torch.cuda.synchronize()
        t = []
        for k in range(args.steps):
            c, st = mcr.forward(med, src, mcr.Run(K=K, n_packets=args.packets, seed=2 + k, sectors=M), stats=True)
            t.append(mcr.last_run_info("forward")[1])
        seg_rate = st["segments"] / (float(np.mean(t)) * 1e-3)
        # spread over 8 seeds of a^(1e6 packets): channel 0 (fluence) for harmonics, sector 0 for M
        vals = np.array([mcr.forward(med, src, mcr.Run(K=K, n_packets=1_000_000, seed=100 + k, sectors=M))
                         [:, pix[0], pix[1]].double().cpu().numpy() for k in range(8)])
        rel = vals.std(axis=0, ddof=1) / np.abs(vals.mean(axis=0))
        C = M if M else 2 * K + 1
        words = (C + 15) // 16 * 16 if C > 32 else (C + 3) // 4 * 4
        rows.append({"tally": label, "K": K, "sectors": M, "channels": C, "tally_words_per_pixel": words,
                     "transport_ms": float(np.mean(t)), "segments_per_s": seg_rate,
                     "photons_per_s": args.packets / (float(np.mean(t)) * 1e-3),
                     "rel_spread_fluence_or_first_sector": float(rel[0])})
    out = {"metric": "forward transport photons/s, harmonic vs discrete-ordinates tally", "value":
           rows[-1]["photons_per_s"], "unit": "photons/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
           "ms_per_step": rows[-1]["transport_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
           "config": {"workload": f"sectors: grad256 medium and line source, forward, {args.packets:.0e} packets; "
                                  f"spread over 8 seeds of 1e6 packets at pixel {pix}", "rows": rows},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


def _invert_rect(args):
    """The reconstructions of Sec. 6 on its rectangular-inclusion domain (workloads.rect_phantom):
    --unknown mua: mu_a only (mu_s known), gradient descent with the Hager-Zhang line search and
    the Eq. 29 stop at 1e-9 (Sec. 6.1); --unknown mus: mu_s only (mu_a known), backtracking with
    the sufficient-decrease constant 0.2 of Eq. 30, steps kept in [1e5, 1e9] and a 1e-5 stop
    (Sec. 6.2).  K = 10, --packets
    per MC run (the paper used 1e8), H^meas from 1e8 packets with seed 1001, homogeneous
    background start.  Reports the mean relative error after every accepted step."""
    import torch
    from paper_1608_05238_gb300 import _build, mcr, workloads
    from paper_1608_05238_gb300.autograd import MCSpec, forward_coefficients
    from paper_1608_05238_gb300.inversion import invert, mean_relative_error
    _build.build()
    n_pk = args.packets
    mua_t, mus_t, g, srcs = workloads.rect_phantom()
    dx = float(np.float32(0.05))
    g = float(np.float32(g))
    dev = torch.device("cuda")
    mua_t, mus_t = torch.from_numpy(mua_t).to(dev), torch.from_numpy(mus_t).to(dev)
    sources = [mcr.Source(**s) for s in srcs]
    med_t = mcr.Medium(mua_t, mus_t, dx, g)
    Hmeas = mcr.h_eps(med_t, forward_coefficients(med_t, MCSpec(dx=dx, g=g, sources=sources, K=0,
                                                                 n_packets=100_000_000, seed=1001)))
    spec = MCSpec(dx=dx, g=g, sources=sources, K=10, n_packets=n_pk)
    if args.unknown == "mua":
        start = torch.full_like(mua_t, 0.01)
        kw = dict(unknowns=("mua",), tol=1e-9, line_search="hager_zhang", mua_true=mua_t)
        x0, fixed = start, mus_t
        run = lambda iters: invert(x0, fixed, Hmeas, spec, iters=iters, **kw)
        err0 = mean_relative_error(start, mua_t)
    else:
        start = torch.full_like(mus_t, 5.0)
        kw = dict(unknowns=("mus",), tol=1e-5, line_search="backtracking", armijo=0.2, shrink=0.5,
                  step_bounds=(1e5, 1e9), mus_true=mus_t)
        run = lambda iters: invert(mua_t, start, Hmeas, spec, iters=iters, **kw)
        err0 = mean_relative_error(start, mus_t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = run(args.iters)
    torch.cuda.synchronize()
    T = time.perf_counter() - t0
    key = "rel_err_mua" if args.unknown == "mua" else "rel_err_mus"
    hist = [{"it": h.it, "eps": h.eps, "step": h.step, "mc_evals": h.trials, key: getattr(h, key),
             "seconds": h.seconds} for h in res.history]
    final = getattr(res.history[-1], key) if res.history else err0
    # inside the reconstructed map's inclusion: its mean value and mean relative error
    est, true = (res.mua, mua_t) if args.unknown == "mua" else (res.mus, mus_t)
    incl = true > true.min()
    inclusion = {"true": float(true[incl].mean()), "start": float(start[incl].mean()),
                 "estimate_mean": float(est[incl].mean()),
                 "rel_err_start": mean_relative_error(start[incl], true[incl]),
                 "rel_err": mean_relative_error(est[incl], true[incl])}
    out = {"metric": f"{args.unknown} reconstruction (Sec. 6): mean relative error", "value": final,
           "unit": "relative error", "n_gpus": 1, "steps": len(res.history), "warmup": 0,
           "ms_per_step": 1e3 * T / max(1, len(res.history)), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient)", "data": "synthetic",
           "config": {"workload": f"invert_rect: 80x80 px of 0.05 mm, rectangular inclusions (mu_a 0.01/0.2, "
                                  f"mu_s 5/15), g 0.9, line sources on z=0 and x=4 mm, K=10, {n_pk:.0e} packets "
                                  f"per MC run, " + ("Hager-Zhang GD, tol 1e-9" if args.unknown == "mua"
                                                     else "backtracking GD (Eq. 30 nu 0.2), tol 1e-5"),
                      "initial_rel_err": err0, "inclusion": inclusion, "converged": res.converged, "seconds": T,
                      "history": hist},
           "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    return 0


METRIC3 = "3D gradient evaluation photons/s (forward + adjoint)"


def cpu_oracle_rate3(mua, mus, mua_true, src, dx, g, L, sample, seed):
    """The 3D oracle as it stands on the host cores: one forward and one adjoint run of ``sample``
    packets on the full grid (adjoint source from the true-minus-estimate absorption, the shape
    of a real one).  Returns (photons/s, seconds, segments per photon)."""
    import oracle
    from oracle import RunParams
    m64, s64 = mua.astype(np.float64), mus.astype(np.float64)
    t0 = time.perf_counter()
    fo = oracle.forward3(m64, s64, np.float32(dx), np.float32(g), src, RunParams(K=L, n_packets=sample, seed=seed))
    qo = (-m64 * (m64 - mua_true) / dx ** 3).astype(np.float32)
    ao = oracle.adjoint3(m64, s64, np.float32(dx), np.float32(g), qo, RunParams(K=L, n_packets=sample, seed=seed + 1))
    dt = time.perf_counter() - t0
    return 2 * sample / dt, dt, {"forward_segments": fo.stats["segments"] / sample,
                                 "adjoint_segments": ao.stats["segments"] / sample}


def _reference3(args):
    """--impl reference for grad3d: the 3D oracle on the host cores, the same metric and config."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1608_05238_gb300 import workloads
    n, L, dx, g = args.n3, args.l3, 0.1, 0.9
    mua, mus, mua_true, src = workloads.phantom3(n, dx, seed=0)
    sample = max(4000, args.cpu_sample // 10)
    for k in range(args.warmup):
        cpu_oracle_rate3(mua, mus, mua_true, src, dx, g, L, sample // 4, seed=10 * k)
    T = 0.0
    for k in range(args.steps):
        _, dt, _ = cpu_oracle_rate3(mua, mus, mua_true, src, dx, g, L, sample, seed=100 + 10 * k)
        T += dt
    value = 2 * sample * args.steps / T
    desc = f"{sample} forward + {sample} adjoint packets per step of grad3d (full {n}^3 grid, L={L})"
    out = {"impl": "reference", "metric": METRIC3, "value": value, "unit": "photons/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"grad3d: {n}^3 voxels of {dx} mm, L={L}, g={g}, pencil beam"},
           "cpu_baseline": {"value": value, "unit": "photons/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": "photons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _grad3d(args):
    """The 3D gradient evaluation (spherical-harmonic tallies): forward run from the pencil beam,
    H and dL/dH against a synthetic measurement, q*, adjoint run, and the voxel gradients, on the
    n^3 phantom; photons (forward + adjoint) per second, the transport's payload rate, and the
    FP64 oracle's rate on a sample of the same runs."""
    import torch
    from paper_1608_05238_gb300 import _build, mcr, mcr3, workloads
    _build.build()
    n, L, dx, g = args.n3, args.l3, 0.1, 0.9
    mua, mus, mua_true, src = workloads.phantom3(n, dx, seed=0)
    dev = lambda a: torch.from_numpy(a).cuda()
    med = mcr3.Medium3(dev(mua), dev(mus), dx, g)
    s3 = mcr3.Source3(**src)
    N = args.packets  # 1e7 forward + 1e7 adjoint packets per step by default
    Hm = mcr3.h_eps(mcr3.Medium3(dev(mua_true), dev(mus), dx, g),
                    mcr3.forward(mcr3.Medium3(dev(mua_true), dev(mus), dx, g), s3, mcr.Run(K=0, n_packets=4 * N,
                                                                                             seed=999)))
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def step(k):
        c, sf = mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N, seed=2 * k), stats=True)
        H, v, eps = mcr3.h_eps(med, c, Hm)
        q = mcr3.adjoint_source(med, v)
        ca, sa = mcr3.adjoint(med, q, mcr.Run(K=L, n_packets=N, seed=2 * k + 1, stream_id=1), stats=True)
        return mcr3.gradient(med, c, ca, v), sf, sa

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    T, segs = 0.0, []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, sf, sa = step(100 + k)
        b.record()
        b.synchronize()
        T += a.elapsed_time(b) * 1e-3
        segs += [sf["segments"], sa["segments"]]
    clocks = clk.stop()
    # the transport alone: one forward run timed by events around the call (its memsets, medium
    # check and finalize included)
    tr = []
    for k in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, st = mcr3.forward(med, s3, mcr.Run(K=L, n_packets=N, seed=500 + k), stats=True)
        b.record()
        b.synchronize()
        tr.append((a.elapsed_time(b), st["segments"]))
    C = (L + 1) ** 2
    ms = float(np.mean([t for t, _ in tr]))
    seg = float(np.mean([s for _, s in tr]))
    achieved = C * 8 * seg / (ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # DRAM bytes per forward launch: 21.05 GB at 1e6 packets (ncu, 96^3, L = 4), scaled by packets
    traffic = 21.05e9 * N / 1e6 if (n, L) == (96, 4) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_transport3", "launch_ms": ms, "segments_per_launch": seg,
                "bytes_per_segment": C * 8,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}
    if not args.no_red_probe:
        red = l2_reduction_peak(n ** 3, C, row_words=(C + 15) // 16 * 16 if C > 16 else (C + 3) // 4 * 4)
        roofline["l2_reduction_peak"] = dict(red, frac=achieved / red["value"])
    value = 2 * N * args.steps / T
    cpu = None
    if not args.no_cpu_baseline:
        sample = max(4000, args.cpu_sample // 10)
        rate, dt, work = cpu_oracle_rate3(mua, mus, mua_true, src, dx, g, L, sample, seed=1)
        cpu = {"value": rate, "unit": "photons/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{sample} forward + {sample} adjoint packets of grad3d (full grid, L={L}), {dt:.1f} s",
               "work_per_photon": work}
    out = {"metric": METRIC3, "value": value, "unit": "photons/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64 (FP64 gradient)",
           "data": "synthetic",
           "config": {"workload": f"grad3d: {n}^3 voxels of {dx} mm, L={L} ({C} channels), g={g}, pencil beam, "
                                  f"{N:.0e} forward + {N:.0e} adjoint packets per step",
                      "segments_per_photon": float(np.mean(segs)) / N, "l2": "flushed between timed steps (256 MB write)"},
           "clocks": clocks, "gpu_launches": 14 * args.steps, "roofline": roofline, "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)
    return 0


def replace_spec(spec, **kw):
    from dataclasses import replace
    return replace(spec, **kw)


def main():
    args = _args()
    if args.workload == "invert256" and args.impl != "reference":
        return _invert256(args)
    if args.workload == "batch64" and args.impl != "reference":
        return _batch64(args)
    if args.workload == "denoise256" and args.impl != "reference":
        return _denoise256(args)
    if args.workload == "conv" and args.impl != "reference":
        return _conv_only(args)
    if args.workload == "unet256" and args.impl != "reference":
        return _unet256(args)
    if args.workload == "invert_rect" and args.impl != "reference":
        return _invert_rect(args)
    if args.workload == "equal_error" and args.impl != "reference":
        return _equal_error(args)
    if args.workload == "invert1024" and args.impl != "reference":
        return _invert1024(args)
    if args.workload == "sectors" and args.impl != "reference":
        return _sectors(args)
    if args.workload == "grad3d" and args.impl != "reference":
        return _grad3d(args)
    if args.impl == "reference":
        return _reference3(args) if args.workload == "grad3d" else _reference(args)
    return _gpu(args)


if __name__ == "__main__":
    sys.exit(main())
