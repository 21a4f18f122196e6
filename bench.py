#!/usr/bin/env python
"""Benchmark of the explicit FD sweep on B300 through the C ABI.

Default workload (one GPU): a 3-D acoustic shot, 256³ FP32 grid (dx = 10 m,
40-point damping layer inside it), space order 8, layered velocity 1.5-4.5 km/s
with 5% smoothed noise, CFL dt, a 10 Hz Ricker source at the centre and a line
of 256 receivers, 500 time steps.  One benchmark *step* is one whole shot:
coefficient setup from m and damp, field reset, 500 time steps (stencil,
injection, interpolation).  ``value`` is grid-point updates per second (GPts/s)
with every input already resident in HBM; ``e2e`` is the same metric through
the C ABI with pinned host buffers (host->device copies of the shot's inputs and
the device->host read of its traces inside the timed region).

``--workload roofline512 --so {4,8,12,16}`` runs the 512³ sweep (200 steps, one
source, no receivers).  ``--workload fwi320`` times full-waveform-inversion
gradients of a 320³, so 8, 1000-step shot (256 receivers) against traces of a
seeded perturbed model: forward sweep with checkpoints every k steps (k tuned
by timing the candidates), recompute, adjoint and imaging per step.  ``--workload serving`` serves a seeded Poisson stream of
64 shots (2-D 200²-1000² and 3-D 128³-320³ grids, so 8, 300-1000 steps, one
source and 128-512 receivers each) with the continuous-batching server under an
HBM budget, and the same stream one shot at a time; it reports shots/s and
p50/p99 latency for both.  ``--impl reference`` times the FP64 CPU oracle on the
same workload instead (a bounded sample of time steps per step).

Multi-GPU (torchrun): shots are independent, so each rank runs its own shot on
its own GPU with no collective in the data path (weak scaling); ranks meet only
at the barriers around the timed region, and the slowest rank's time counts.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fdsynth  # noqa: E402

BYTES_PER_POINT = {"acoustic": 20,   # read u^n, u^{n-1}, A, C; write u^{n+1} (FP32)
                   "diffusion": 8}   # read u^n, write u^{n+1}
FALLBACK_HBM_GBS = 6400.0

WORKLOADS = {
    "acoustic256": dict(n=256, so=8, nt=500, nrec=256, nbl=40),
    "roofline512": dict(n=512, so=8, nt=200, nrec=0, nbl=40),
    # the largest 2-D shot of the serving stream: 1000², so 8, 1000 steps, 512 receivers
    # (a level is 4 MB: the fields stay in L2, so HBM is not the bound)
    "acoustic2d": dict(n=1000, so=8, nt=1000, nrec=512, nbl=40, ndim=2),
}

# DRAM bytes per stencil launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, mean of the captured launches; the captures with ncu's default
# L2 flush count only the writes that leave L2 during the launch, the warm capture also
# the previous step's write-backs), keyed by (kernel name,
# workload, space order, tile width, tile height, z-block height, CTAs per SM, aligned,
# skip_c); the captures
# are summarised in profiles/.  Absent (null) when not captured for the kernel
# and tile configuration as they are now.
NCU_TRAFFIC = {
    # profiles/stencil3d_tma_acoustic256_so8.md ("Warm-L2 DRAM traffic"): the 32-wide kernel
    # (32 x 32 tiles, 2 CTAs/SM, 64-plane segments), L2 not flushed between launches (the
    # bench's conditions): mean of 3 launches, read 260.47 MB + write 68.50 MB
    ("stencil3d_tma_acoustic", "acoustic256", 8, 32, 32, 64, 2, 1, 0): 328.97e6,
    # same section, the x-pair kernel (64 x 32 tiles, 1 CTA/SM): read 260.04 MB + write 66.80 MB
    ("stencil3d_xp_acoustic", "acoustic256", 8, 64, 32, 64, 1, 1, 0): 326.84e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="acoustic256",
                    choices=sorted(WORKLOADS) + ["serving", "fwi320", "diffusion512",
                                                 "diffusion2d"])
    ap.add_argument("--boundary", default="zero", choices=["zero", "odd"],
                    help="diffusion512: values outside the grid (zero halo or odd reflection)")
    ap.add_argument("--fwi-k", type=int, default=0,
                    help="fwi320: checkpoint interval (0: tuned by timing the candidates)")
    ap.add_argument("--shots", type=int, default=64)
    ap.add_argument("--mean-gap", type=float, default=0.015)
    ap.add_argument("--hbm-budget-gb", type=float, default=8.0)
    ap.add_argument("--work-cap", type=int, default=65_000_000,
                    help="serving: most grid points one batch tick updates (0: no cap); "
                         "65 M (about four 256^3 shots) keeps the GPU saturated while a "
                         "long shot is not stretched by everything admitted beside it")
    ap.add_argument("--ticks-per-round", type=int, default=32,
                    help="serving: most batch steps between admission points")
    ap.add_argument("--so", type=int, default=None)
    ap.add_argument("--n", type=int, default=None,
                    help="acoustic workloads: grid points per axis instead of the workload's")
    ap.add_argument("--nt", type=int, default=None)
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tma"])
    ap.add_argument("--tile", default="auto",
                    help="auto: the autotuner picks the pipelined kernel's tile configuration "
                         "before the timed region; default: the built-in one; "
                         "TY,ZB,CPS[,AL[,SK[,TX]]]: tile height (16, 32; 24 with TX 64 from "
                         "so 8), z-block height, CTAs per SM, split (0 equal ranges, 1 whole "
                         "segments, 2 work queue with TX 64), C-tile skipping and tile width "
                         "(64: the x-pair kernel) given explicitly")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extras", default="sweep512,serving,fwi320,c1,diffusion2d,oracle",
                    help="default workload, one GPU: legs measured after the main timed region "
                         "and added to its line (comma list; empty for none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def problem(args):
    w = dict(WORKLOADS[args.workload])
    if args.so:
        w["so"] = args.so
    if args.n:
        w["n"] = args.n
        w["nbl"] = min(w["nbl"], max(4, args.n // 8))
    if args.nt:
        w["nt"] = args.nt
    p = fdsynth.acoustic_problem(n=w["n"], ndim=w.get("ndim", 3), so=w["so"], nbl=w["nbl"],
                                 nt=w["nt"], nrec=w["nrec"], seed=0)
    return w, p


def config_of(args, w, kernel_name=None):
    nd = w.get("ndim", 3)
    cfg = {"workload": f"acoustic{nd}d_{w['n']}^{nd}_so{w['so']}_nt{w['nt']}",
           "grid": [w["n"]] * nd, "space_order": w["so"], "nt": w["nt"], "nrec": w["nrec"],
           "nsrc": 1, "damping_layer": w["nbl"], "dx_m": 10.0,
           "step": "one shot: coefficient setup + field reset + nt time steps",
           "l2": ("inputs larger than L2 (u^n, u^{n-1}, A, C = 4 x %.0f MB)" %
                  ((w["n"] + 8) ** 2 * (w["n"] + 64) * 4 / 1e6)) if nd == 3 else
                 ("fields L2-resident (4 levels of %.1f MB): the per-launch time is bound by "
                  "L2 bandwidth and launch latency, not HBM" %
                  ((w["n"] + 8) * (w["n"] + 64) * 4 / 1e6))}
    if kernel_name:
        cfg["kernel"] = kernel_name
    return cfg


def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x):
    """Maximum of a float over all ranks (identity without torch.distributed).

    Works with NCCL (CUDA tensor) and gloo (CPU tensor) process groups."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Aggregate throughput: every rank processed units_per_rank in the slowest rank's time."""
    return world * units_per_rank / seconds


def cpu_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def time_oracle(p, steps):
    """Oracle GPts/s over `steps` time steps of the shot (source and receivers included)."""
    from oracle import core as oracle
    m = p["m"].astype(np.float64)
    damp = p["damp"].astype(np.float64)
    rec = p["rec_coords"] if len(p["rec_coords"]) else None
    t0 = time.perf_counter()
    oracle.acoustic(m, p["dt"], p["spacing"], p["so"], steps, damp=damp,
                    src_coords=p["src_coords"], wavelet=p["wavelet"], rec_coords=rec)
    dt = time.perf_counter() - t0
    return m.size * steps / dt / 1e9, dt


def oracle_steps_for(p, budget_s):
    """Time steps of the oracle that fill about budget_s seconds (a call has a fixed
    set-up cost, so the per-step time comes from a 1-step and a 3-step call)."""
    _, t1 = time_oracle(p, 1)
    _, t3 = time_oracle(p, 3)
    per = max((t3 - t1) / 2.0, 1e-4)
    setup = max(t1 - per, 0.0)
    return int(max(1, min(p["nt"], round((budget_s - setup) / per))))


def cpu_baseline(p, budget_s):
    k = oracle_steps_for(p, budget_s)
    v, t = time_oracle(p, k)
    if t < 0.5 * budget_s and k < p["nt"]:
        # the 1- and 3-step calls misjudged the per-step time (page faults, thread
        # start-up): one more sample, scaled by what this one took
        k = int(min(p["nt"], max(k + 1, round(k * budget_s / max(t, 1e-3)))))
        v, t = time_oracle(p, k)
    return {"value": round(v, 4), "unit": "GPts/s", "cores": cpu_threads(), "kind": "oracle",
            "sample": f"first {k} of {p['nt']} time steps of the same shot (FP64, "
                      f"{t:.1f} s), OpenMP over grid rows"}


def run_reference_fwi(args):
    """Reference arm of the FWI workload: the FP64 oracle gradient on a bounded sample."""
    w, _ = fwi_problem(args)
    for _ in range(args.warmup):
        fwi_oracle_sample(0.0)
    vals, sample = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, sample = fwi_oracle_sample(0.0)
        vals.append(v)
    total = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": "FWI gradient GPts/s (space-time points of the shot per second)",
            "value": round(value, 5), "unit": "GPts/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": fwi_config(w),
            "cpu_baseline": {"value": round(value, 5), "unit": "GPts/s", "cores": cpu_threads(),
                             "kind": "oracle", "sample": "each step = " + sample},
            "e2e": {"value": round(value, 5), "unit": "GPts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    if args.workload == "fwi320":
        return run_reference_fwi(args)
    if args.workload in ("serving", "diffusion512", "diffusion2d"):
        args.workload = "acoustic256"     # the oracle's timed sample: the acoustic shot
    w, p = problem(args)
    per_step = oracle_steps_for(p, 6.0)
    for _ in range(args.warmup):
        time_oracle(p, per_step)
    vals, total = [], 0.0
    for _ in range(args.steps):
        v, t = time_oracle(p, per_step)
        vals.append(v)
        total += t
    value = (p["m"].size * per_step * args.steps) / total / 1e9
    line = {"impl": "reference", "metric": "GPts/s & % HBM roofline per stencil", "value": round(value, 4),
            "unit": "GPts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, w),
            "cpu_baseline": {"value": round(value, 4), "unit": "GPts/s", "cores": cpu_threads(),
                             "kind": "oracle",
                             "sample": f"each step = first {per_step} of {p['nt']} time steps of the shot"},
            "e2e": {"value": round(value, 4), "unit": "GPts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


FWI = dict(n=320, so=8, nt=1000, nrec=256, nbl=40)
# algorithmic bytes per grid point and time step of one gradient, by backward sweep:
#   fused (fd_step_fwi): forward 20 + recompute writing d2 24 + adjoint with imaging 32
#   separate kernels: forward 20 + recompute 20 + snapshot 8 + adjoint 20 + imaging 24
FWI_BYTES_PER_POINT_STEP = {True: 76, False: 92}
FWI_STENCIL_BYTES = {True: 76, False: 60}   # of those, moved by the 3 stencil launches


def fwi_problem(args):
    w = dict(FWI)
    if args.nt:
        w["nt"] = args.nt
    p = fdsynth.acoustic_problem(n=w["n"], ndim=w.get("ndim", 3), so=w["so"], nbl=w["nbl"],
                                 nt=w["nt"], nrec=w["nrec"], seed=0)
    return w, p


def fwi_config(w, k=None, tuning=None):
    cfg = {"workload": f"fwi_gradient_acoustic3d_{w['n']}^3_so{w['so']}_nt{w['nt']}",
           "grid": [w["n"]] * 3, "space_order": w["so"], "nt": w["nt"], "nrec": w["nrec"],
           "nsrc": 1, "damping_layer": w["nbl"], "dx_m": 10.0,
           "step": "one gradient dJ/dm: forward with checkpoints, recompute, adjoint, imaging",
           "observed_data": "traces of a seeded perturbed model (4 Gaussian blobs, +5% in m)",
           "l2": "inputs larger than L2 (each level %.0f MB)" %
                 ((w["n"] + 8) ** 2 * (w["n"] + 64) * 4 / 1e6)}
    if k is not None:
        cfg["checkpoint_interval"] = k
    if tuning is not None:
        cfg["checkpoint_tuning"] = tuning
    return cfg


def fwi_oracle_sample(budget_s):
    """Oracle gradient GPts/s on a bounded sample: 40³ grid of the same recipe."""
    from oracle import fwi as ofwi
    n, nt = 40, 60
    q = fdsynth.acoustic_problem(n=n, ndim=3, so=8, nbl=8, nt=nt, nrec=64, seed=0)
    m_true = fdsynth.perturbed_model(q["m"], 8)
    from oracle import core as oracle
    _, _, d_obs = oracle.acoustic(m_true, q["dt"], q["spacing"], 8, nt, damp=q["damp"],
                                  src_coords=q["src_coords"], wavelet=q["wavelet"],
                                  rec_coords=q["rec_coords"])
    runs, total = 0, 0.0
    while total < budget_s or runs == 0:
        t0 = time.perf_counter()
        ofwi.gradient(q["m"], q["damp"], q["dt"], q["spacing"], 8, nt, q["src_coords"],
                      q["wavelet"], q["rec_coords"], d_obs)
        total += time.perf_counter() - t0
        runs += 1
    value = n ** 3 * nt * runs / total / 1e9
    return value, f"{runs} FP64 oracle gradients of a 40^3, so 8, 60-step shot of the same recipe ({total:.1f} s)"


def fwi_result(args, world=1, rank=0, local=0):
    """Whole FWI gradients of the 320³ shot, timed: the result line."""
    import torch
    from paper_1906_10811_b300 import build, fwi
    build.build()
    w, p = fwi_problem(args)
    npts, nt = int(np.prod(p["shape"])), p["nt"]
    m_true = fdsynth.perturbed_model(p["m"], w["nbl"])
    d_obs = fwi.forward_traces(p, m_true)
    m0 = torch.from_numpy(p["m"]).cuda()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    tuning = None
    if args.fwi_k > 0:
        k = args.fwi_k
    else:
        k, rows = fwi.tune_checkpoint_interval(p, d_obs, m=m0)
        tuning = [{"k": r[0], "s": round(r[1], 4), "bytes": int(r[2])} for r in rows]
    stats = {}
    for _ in range(args.warmup):
        fwi.gradient(p, d_obs, m=m0, k=k, stats=stats)
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    clocks = ClockSampler(gpu_id)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        st = {}
        fwi.gradient(p, d_obs, m=m0, k=k, stats=st)
        launches += st["launches_forward"] + st["launches_adjoint"]
    e1.record(stream)
    barrier()
    ms = reduce_max(e0.elapsed_time(e1))
    clk = clocks.stop()
    value = whole_job_rate(npts * nt * args.steps, world, ms / 1e3) / 1e9

    # stencil launches timed one by one (outside the timed region)
    prof = {}
    fwi.gradient(p, d_obs, m=m0, k=k, stats=prof, profile=True)
    fused = bool(prof.get("fused"))
    avg_s = prof["stencil_ms"] / max(prof["stencil_launches"], 1) / 1e3
    peak, peak_kind = load_peak()
    per_launch_b = FWI_STENCIL_BYTES[fused] / 3.0        # mean over forward, recompute, adjoint
    achieved = per_launch_b * npts / avg_s / 1e9
    grad_b = FWI_BYTES_PER_POINT_STEP[fused]
    grad_gbs = grad_b * npts * nt * args.steps / (ms / 1e3) / 1e9 / world
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "stencil3d_tma_acoustic (forward; recompute and adjoint with the "
                          "FWI epilogue)" if fused else "stencil3d_tma_acoustic",
                "bytes_per_point": round(per_launch_b, 3), "points_per_launch": npts,
                "avg_launch_us": round(avg_s * 1e6, 2),
                "launches_timed": prof["stencil_launches"],
                "stencil_share_of_step": round(prof["stencil_ms"] / (ms / args.steps), 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})",
                "whole_gradient": {"bytes_per_point_step": grad_b, "fused_backward": fused,
                                   "achieved_gbs": round(grad_gbs, 1),
                                   "frac": round(grad_gbs / peak, 4)}}

    e2e = None
    if not args.no_e2e:
        m_h = torch.from_numpy(p["m"]).pin_memory()
        d_h = d_obs.cpu().pin_memory()
        g_h = torch.empty(p["shape"], dtype=torch.float32).pin_memory()

        def grad_e2e():
            m_d = m_h.cuda(non_blocking=True)
            d_d = d_h.cuda(non_blocking=True)
            _, g = fwi.gradient(p, d_d, m=m_d, k=k)
            g_h.copy_(g, non_blocking=True)

        grad_e2e()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            grad_e2e()
        barrier()
        te = reduce_max(time.perf_counter() - t0)
        e2e = {"value": round(whole_job_rate(npts * nt * args.steps, world, te) / 1e9, 3),
               "unit": "GPts/s", "h2d_bytes_per_step": int(m_h.numel() * 4 + d_h.numel() * 4),
               "d2h_bytes_per_step": int(g_h.numel() * 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample = fwi_oracle_sample(args.cpu_seconds)
        cpu = {"value": round(v, 5), "unit": "GPts/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": sample}
    line = {"metric": "FWI gradient GPts/s (space-time points of the shot per second)",
            "value": round(value, 3), "unit": "GPts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(fwi_config(w, k, tuning),
                           checkpoint_bytes=stats.get("checkpoint_bytes"),
                           block_bytes=stats.get("block_bytes"), tile=stats.get("tile"),
                           tile_choice="fd_autotune_fwi (plain + d2 + imaging steps)"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk}
    return line


def run_fwi(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = fwi_result(args, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_diffusion(args):
    """Diffusion sweep: 3-D at 512³ (sine-mode data, ν dt/h² = 0.05, interior update), or
    with --workload diffusion2d the paper's benchmark problem (§5.1.2): 2-D sine-mode
    data with ν = 0.5 on n² nodes (default 10000², a size the paper measured), ν dt/h² =
    0.1 (stable up to so 16), interior update."""
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1906_10811_b300 import Solver, build
    build.build()
    two = args.workload == "diffusion2d"
    nd = 2 if two else 3
    n, so, nt = (args.n or (10000 if two else 512)), args.so or 8, args.nt or 200
    q = fdsynth.diffusion_problem(n, ndim=nd, courant=0.1 if two else 0.05)
    npts = n ** nd
    u0_d = torch.from_numpy(q["u0"]).cuda()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    bench_stream = torch.cuda.Stream()
    bench_stream.wait_stream(torch.cuda.current_stream())
    torch.cuda.set_stream(bench_stream)
    s = Solver((n,) * nd, q["spacing"], so, q["dt"], "diffusion", nu=q["nu"], device=True,
               profile=True, kernel=args.kernel, boundary=args.boundary)
    tile, tune_tried = None, None
    if s.kernel_name.startswith(("stencil3d_tma", "stencil3d_xp")):
        s.set_field(u0_d)
        if args.tile == "auto":
            tune_tried = len(s.autotune(reps=5)[1])
        elif args.tile != "default":
            ty, zb, cps, al, sk, tx = ([int(v) for v in args.tile.split(",")] + [0, 0, 0])[:6]
            s.set_tile_config(tile_y=ty, zblock=zb, ctas_per_sm=cps, aligned=al, skip_c=sk,
                              tile_x=tx)
        tile = s.tile_config

    def sweep():
        s.set_field(u0_d)
        s.set_step(0)
        s.run(nt)

    for _ in range(args.warmup):
        sweep()
    s.profile()
    launches0 = s.kernel_launches
    clocks = ClockSampler("GPU-" + str(torch.cuda.get_device_properties(local).uuid))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        sweep()
    e1.record(stream)
    barrier()
    ms = reduce_max(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = s.kernel_launches - launches0
    n_st, st_ms = s.profile()
    kernel_name = s.kernel_name
    s.close()
    value = whole_job_rate(npts * nt * args.steps, world, ms / 1e3) / 1e9
    peak, peak_kind = load_peak()
    avg_s = st_ms / max(n_st, 1) / 1e3
    achieved = BYTES_PER_POINT["diffusion"] * npts / avg_s / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": kernel_name,
                "bytes_per_point": BYTES_PER_POINT["diffusion"], "points_per_launch": npts,
                "avg_launch_us": round(avg_s * 1e6, 2), "launches_timed": n_st,
                "stencil_share_of_step": round(st_ms / ms, 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})",
                "gpts_per_s_kernel": round(npts / avg_s / 1e9, 2)}
    if kernel_name == "stencil2d_stream2":
        # two steps a launch: the profile counts steps, so the figures above are per
        # step at the algorithmic 8 B per point-step; the launch moves 4 per point-step
        roofline["bytes_moved_per_point_step"] = BYTES_PER_POINT["diffusion"] / 2
        roofline["note"] = ("two steps a launch: per-step time at the algorithmic 8 B per "
                            "point-step; each launch reads u^n and writes u^{n+2} once")
    e2e = None
    if not args.no_e2e:
        u0_h = torch.from_numpy(q["u0"]).pin_memory().numpy()
        out_h = torch.empty((n,) * nd, dtype=torch.float32).pin_memory().numpy()
        se = Solver((n,) * nd, q["spacing"], so, q["dt"], "diffusion", nu=q["nu"],
                    kernel=args.kernel, boundary=args.boundary)
        if tile is not None:
            se.set_tile_config(tile_y=tile["tile_y"], zblock=tile["zblock"],
                               ctas_per_sm=tile["ctas_per_sm"], aligned=tile["aligned"],
                               skip_c=tile["skip_c"], tile_x=tile["tile_x"])
        from paper_1906_10811_b300 import binding as B

        def sweep_e2e():
            se.set_field(u0_h)
            se.set_step(0)
            se.run(nt)
            B.fd_read(se.ctx, out_h, None)

        sweep_e2e()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sweep_e2e()
        barrier()
        te = reduce_max(time.perf_counter() - t0)
        se.close()
        e2e = {"value": round(whole_job_rate(npts * nt * args.steps, world, te) / 1e9, 3),
               "unit": "GPts/s", "h2d_bytes_per_step": int(u0_h.nbytes),
               "d2h_bytes_per_step": int(out_h.nbytes)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import core as oracle
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < args.cpu_seconds or k == 0:
            oracle.diffusion(q["u0"], q["spacing"], so, q["nu"], q["dt"], 1,
                             boundary=args.boundary)
            k += 1
        tc = time.perf_counter() - t0
        cpu = {"value": round(npts * k / tc / 1e9, 4), "unit": "GPts/s", "cores": cpu_threads(),
               "kind": "oracle", "sample": f"{k} single time steps of the same 512^3 sweep "
                                           f"(FP64, {tc:.1f} s), OpenMP over grid rows"}
    if rank == 0:
        line = {"metric": "GPts/s & % HBM roofline per stencil", "value": round(value, 3),
                "unit": "GPts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"diffusion{nd}d_{n}^{nd}_so{so}_nt{nt}", "grid": [n] * nd,
                           "space_order": so, "nt": nt, "nu": q["nu"],
                           "nu_dt_over_h2": 0.1 if two else 0.05, "boundary": args.boundary,
                           "initial_data": "product of sin(pi x_d), boundary nodes 0",
                           "step": "one sweep: field reset + nt time steps",
                           "l2": "inputs larger than L2 (u^n, u^{n+1} = 2 x %.0f MB)" %
                                 ((n + so) ** (nd - 1) * (n + 64) * 4 / 1e6),
                           "kernel": kernel_name, "tile": tile,
                           "tile_choice": ("autotuned over %d configurations" % tune_tried
                                           if tune_tried else args.tile)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


SWEEP_ORDERS = (4, 8, 12, 16)


def _gpu_uuid():
    import torch
    return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)


def sweep512_result(reps=2, orders=SWEEP_ORDERS):
    """512³ roofline sweep on the current torch stream: per space order the autotuned
    tile, µs per stencil launch (graph-chunk events), the fraction of the measured HBM
    copy bandwidth at the algorithmic bytes per point, and GPts/s of whole shots
    (acoustic: coefficient set-up, reset and 200 steps with one source; diffusion:
    field reset and 200 steps of the sine-mode problem at ν dt/h² = 0.05)."""
    import torch
    from paper_1906_10811_b300 import Solver
    n, nt = 512, 200
    npts = n ** 3
    peak, peak_kind = load_peak()
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def measure(s, shot, bpp):
        shot()
        s.profile()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            shot()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        n_st, st_ms = s.profile()
        avg = st_ms / max(n_st, 1) / 1e3
        ach = bpp * npts / avg / 1e9
        t = s.tile_config
        return {"us_per_launch": round(avg * 1e6, 2), "achieved_gbs": round(ach, 1),
                "frac": round(ach / peak, 4), "gpts_per_s_kernel": round(npts / avg / 1e9, 2),
                "gpts_per_s_shot": round(npts * nt * reps / (ms / 1e3) / 1e9, 2),
                "kernel": s.kernel_name,
                "tile": {k: t[k] for k in ("tile_x", "tile_y", "zblock", "ctas_per_sm",
                                           "aligned", "skip_c")}}

    clocks = ClockSampler(_gpu_uuid())
    p = fdsynth.acoustic_problem(n=n, ndim=3, so=8, nbl=40, nt=nt, nrec=0, seed=0)
    m_d, damp_d = dev(p["m"]), dev(p["damp"])
    src_d, wav_d = dev(p["src_coords"]), dev(p["wavelet"])
    acoustic = {}
    for so in orders:
        s = Solver((n,) * 3, p["spacing"], so, p["dt"], "acoustic", device=True, profile=True)
        s.set_sources(src_d, wav_d)
        s.set_model(m_d, damp_d)
        tried = len(s.autotune(reps=3)[1])

        def shot():
            s.set_model(m_d, damp_d)
            s.reset()
            s.run(nt)

        acoustic[f"so{so}"] = dict(measure(s, shot, BYTES_PER_POINT["acoustic"]),
                                   configs_tried=tried)
        s.close()
    del m_d, damp_d
    torch.cuda.empty_cache()
    q = fdsynth.diffusion_problem(n, ndim=3, courant=0.05)
    u0_d = dev(q["u0"])
    diffusion = {}
    for so in orders:
        s = Solver((n,) * 3, q["spacing"], so, q["dt"], "diffusion", nu=q["nu"], device=True,
                   profile=True)
        s.set_field(u0_d)
        tried = len(s.autotune(reps=3)[1])

        def sweep():
            s.set_field(u0_d)
            s.set_step(0)
            s.run(nt)

        diffusion[f"so{so}"] = dict(measure(s, sweep, BYTES_PER_POINT["diffusion"]),
                                    configs_tried=tried)
        s.close()
    del u0_d
    torch.cuda.empty_cache()
    return {"grid": [n] * 3, "nt": nt, "shots_timed": reps, "acoustic": acoustic,
            "diffusion": diffusion, "peak": peak,
            "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})",
            "bytes_per_point": dict(BYTES_PER_POINT),
            "note": "frac counts the algorithmic bytes per point; with skip_c the undamped "
                    "tile-planes move 16 of the acoustic 20 B/pt",
            "clocks": clocks.stop()}


def diffusion2d_result(n=10000, orders=(2, 4, 8, 16), nt=100, reps=2):
    """The paper's benchmark problem (§5.1.2: 2-D diffusion, sine-mode data, ν = 0.5,
    interior update) at n² = 10000², a size the paper measured: per space order the
    kernel, µs per step (the profile counts steps; the two-step stream at so 2/4 runs
    two a launch), fraction of the measured copy bandwidth at the algorithmic 8 B per
    point-step, the bytes per point-step the kernel actually moves (4 for two steps a
    launch) and GPts/s of whole sweeps (field reset + nt steps)."""
    import torch
    from paper_1906_10811_b300 import Solver
    peak, peak_kind = load_peak()
    stream = torch.cuda.current_stream()
    q = fdsynth.diffusion_problem(n, courant=0.1)
    u0_d = torch.from_numpy(q["u0"]).cuda()
    npts = n * n
    clocks = ClockSampler(_gpu_uuid())
    out = {}
    for so in orders:
        s = Solver((n, n), q["spacing"], so, q["dt"], "diffusion", nu=q["nu"], device=True,
                   profile=True)

        def sweep():
            s.set_field(u0_d)
            s.set_step(0)
            s.run(nt)

        sweep()
        s.profile()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            sweep()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        n_st, st_ms = s.profile()
        avg = st_ms / max(n_st, 1) / 1e3
        ach = BYTES_PER_POINT["diffusion"] * npts / avg / 1e9
        per_launch = 2 if s.kernel_name == "stencil2d_stream2" else 1
        moved = BYTES_PER_POINT["diffusion"] / per_launch
        out[f"so{so}"] = {"kernel": s.kernel_name, "steps_per_launch": per_launch,
                          "us_per_launch": round(avg * per_launch * 1e6, 2),
                          "us_per_step": round(avg * 1e6, 2), "bytes_moved_per_point_step": moved,
                          "achieved_gbs": round(ach, 1), "frac": round(ach / peak, 4),
                          "gpts_per_s_kernel": round(npts / avg / 1e9, 2),
                          "gpts_per_s_sweep": round(npts * nt * reps / (ms / 1e3) / 1e9, 2)}
        s.close()
    del u0_d
    torch.cuda.empty_cache()
    return {"workload": f"diffusion2d_{n}^2_nt{nt}", "nu_dt_over_h2": 0.1,
            "orders": out, "peak": peak,
            "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})",
            "bytes_per_point": BYTES_PER_POINT["diffusion"], "clocks": clocks.stop()}


def c1_result(reps=20):
    """Config 1 on the device: 128² diffusion, so 2, 100 steps (L2-resident, launch-bound):
    latency of one whole run (field upload from device memory, 100 steps, read back)."""
    import torch
    from paper_1906_10811_b300 import Solver
    q = fdsynth.diffusion_problem(128)
    u0_d = torch.from_numpy(q["u0"]).cuda()
    with Solver(q["u0"].shape, q["spacing"], 2, q["dt"], "diffusion", nu=q["nu"],
                device=True) as s:
        out = torch.empty_like(u0_d)
        from paper_1906_10811_b300 import binding as B

        def run():
            s.set_field(u0_d)
            s.set_step(0)
            s.run(100)
            B.fd_read(s.ctx, out, None)

        run()
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            run()
            t.append(time.perf_counter() - t0)
        kname = s.kernel_name
    ms = 1e3 * statistics.median(t)
    return {"workload": "diffusion2d_128^2_so2_nt100", "kernel": kname,
            "ms_per_run_median": round(ms, 4), "us_per_step": round(1e3 * ms / 100, 3),
            "runs": reps, "note": "host-timed: set_field + 100 graph-replayed steps + read "
                                  "(synchronising); 64 KB per level, L2-resident"}


def oracle_legs(p256):
    """The oracle timed on the host: single-threaded on the 256³ shot, on config 1 and on
    the 512³ so 8 step (bounded samples; a subprocess gives the single-thread run its own
    OpenMP runtime)."""
    legs = {}
    code = ("import sys,time,json; sys.path.insert(0, %r); import fdsynth; "
            "from oracle import core as o; "
            "p=fdsynth.acoustic_problem(n=256,ndim=3,so=8,nbl=40,nt=500,nrec=256,seed=0); "
            "k=3; t=time.perf_counter(); "
            "o.acoustic(p['m'],p['dt'],p['spacing'],8,k,damp=p['damp'],src_coords=p['src_coords'],"
            "wavelet=p['wavelet'],rec_coords=p['rec_coords']); "
            "dt=time.perf_counter()-t; print(json.dumps({'steps':k,'s':dt}))" % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        legs["acoustic256_so8_1thread"] = {
            "value": round(256 ** 3 * d["steps"] / d["s"] / 1e9, 5), "unit": "GPts/s", "cores": 1,
            "sample": f"first {d['steps']} of 500 time steps of the 256^3 shot ({d['s']:.1f} s, "
                      f"set-up included)",
            "extrapolated_shot_s": round(d["s"] / d["steps"] * 500, 1)}
    except Exception as e:                                   # pragma: no cover
        legs["acoustic256_so8_1thread"] = {"error": str(e)[:200]}
    from oracle import core as oracle
    q = fdsynth.diffusion_problem(128)
    t0 = time.perf_counter()
    oracle.diffusion(q["u0"], q["spacing"], 2, q["nu"], q["dt"], 100)
    tc = time.perf_counter() - t0
    legs["c1_diffusion128_so2_nt100"] = {"value": round(128 ** 2 * 100 / tc / 1e9, 5),
                                        "unit": "GPts/s", "cores": cpu_threads(),
                                        "seconds": round(tc, 4), "sample": "whole run (100 steps)"}
    p = fdsynth.acoustic_problem(n=512, ndim=3, so=8, nbl=40, nt=200, nrec=0, seed=0)
    k = 3
    t0 = time.perf_counter()
    oracle.acoustic(p["m"], p["dt"], p["spacing"], 8, k, damp=p["damp"],
                    src_coords=p["src_coords"], wavelet=p["wavelet"])
    tc = time.perf_counter() - t0
    legs["c3_acoustic512_so8"] = {"value": round(512 ** 3 * k / tc / 1e9, 5), "unit": "GPts/s",
                                  "cores": cpu_threads(), "sample": f"first {k} of 200 steps "
                                  f"({tc:.1f} s, set-up included)",
                                  "extrapolated_200_steps_s": round(tc / k * 200, 1),
                                  "extrapolated": True}
    return legs


def run_extras(args, line, p256):
    """The rest of the headline metric, measured after the main timed region (one GPU)."""
    import argparse as _ap
    t_start = time.perf_counter()
    extras = [e for e in args.extras.split(",") if e]
    if "sweep512" in extras:
        line["sweep512"] = sweep512_result()
    if "serving" in extras:
        sv = serving_result(args)
        line["serving"] = {k: sv[k] for k in ("serving", "sequential", "speedup_vs_sequential",
                                              "p99_vs_sequential", "gpts_per_s", "pinned_inputs",
                                              "config", "clocks")}
    if "fwi320" in extras:
        ns = _ap.Namespace(**vars(args))
        ns.steps, ns.warmup, ns.nt, ns.no_cpu_baseline = 2, 1, None, True
        fw = fwi_result(ns)
        line["fwi320"] = {"ms_per_gradient": fw["ms_per_step"], "gpts_per_s": fw["value"],
                          "checkpoint_interval": fw["config"].get("checkpoint_interval"),
                          "tile": fw["config"].get("tile"), "roofline": fw["roofline"],
                          "e2e": fw["e2e"], "gradients_timed": ns.steps,
                          "gpu_launches": fw["gpu_launches"], "clocks": fw["clocks"]}
    if "c1" in extras:
        line["c1_diffusion128"] = c1_result()
    if "diffusion2d" in extras:
        line["diffusion2d"] = diffusion2d_result()
    if "oracle" in extras and line.get("cpu_baseline") is not None:
        line["cpu_baseline"]["legs"] = oracle_legs(p256)
    line["extras_seconds"] = round(time.perf_counter() - t_start, 1)


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1906_10811_b300 import Solver, build
    build.build()

    w, p = problem(args)
    npts = int(np.prod(p["shape"]))
    nt = p["nt"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m_d, damp_d = dev(p["m"]), dev(p["damp"])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timed region ----------------
    # one dedicated stream carries the library's work and the timing events
    bench_stream = torch.cuda.Stream()
    bench_stream.wait_stream(torch.cuda.current_stream())
    torch.cuda.set_stream(bench_stream)
    s = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", device=True, profile=True,
               kernel=args.kernel)
    assert s.stream.cuda_stream == bench_stream.cuda_stream
    s.set_sources(dev(p["src_coords"]), dev(p["wavelet"]))
    if w["nrec"]:
        s.set_receivers(dev(p["rec_coords"]))
    tile, tune_tried = None, None
    if s.kernel_name.startswith("stencil3d_tma"):
        if args.tile == "auto":
            s.set_model(m_d, damp_d)
            _, tried = s.autotune(reps=5)
            tune_tried = len(tried)
        elif args.tile != "default":
            ty, zb, cps, al, sk, tx = ([int(v) for v in args.tile.split(",")] + [0, 0, 0])[:6]
            s.set_tile_config(tile_y=ty, zblock=zb, ctas_per_sm=cps, aligned=al, skip_c=sk,
                              tile_x=tx)
        tile = s.tile_config

    def shot():
        s.set_model(m_d, damp_d)
        s.reset()
        s.run(nt)

    for _ in range(args.warmup):
        shot()
    s.profile()                                            # reset the per-launch timers
    launches0 = s.kernel_launches
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    clocks = ClockSampler(gpu_id)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        shot()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = s.kernel_launches - launches0
    n_st, st_ms = s.profile()
    kernel_name = s.kernel_name
    _, rec_dev = s.read(field=False)
    s.close()
    ms = reduce_max(ms)
    value = whole_job_rate(npts * nt * args.steps, world, ms / 1e3) / 1e9

    peak, peak_kind = load_peak()
    avg_launch_s = st_ms / max(n_st, 1) / 1e3
    achieved = BYTES_PER_POINT["acoustic"] * npts / avg_launch_s / 1e9
    tkey = ((tile["tile_x"], tile["tile_y"], tile["zblock"], tile["ctas_per_sm"], tile["aligned"],
             tile["skip_c"]) if tile else (0, 0, 0, 0, 0, 0))
    traffic = NCU_TRAFFIC.get((kernel_name, args.workload, w["so"]) + tkey)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": kernel_name, "bytes_per_point": BYTES_PER_POINT["acoustic"],
                "points_per_launch": npts, "avg_launch_us": round(avg_launch_s * 1e6, 2),
                "launches_timed": n_st, "stencil_share_of_step": round(st_ms / ms, 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})",
                "gpts_per_s_kernel": round(npts / avg_launch_s / 1e9, 2)}

    # ---------------- end to end through the C ABI with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        m_h, damp_h = pin(p["m"]), pin(p["damp"])
        src_h, wav_h, rc_h = pin(p["src_coords"]), pin(p["wavelet"]), pin(p["rec_coords"])
        rec_out = torch.empty((nt + 1, max(w["nrec"], 1)), dtype=torch.float32).pin_memory().numpy()
        h2d = m_h.nbytes + damp_h.nbytes + src_h.nbytes + wav_h.nbytes + rc_h.nbytes
        d2h = (nt + 1) * w["nrec"] * 4
        se = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", device=False,
                    kernel=args.kernel, autotune=tile is not None and args.tile == "auto")
        if tile is not None and args.tile not in ("auto", "default"):
            se.set_tile_config(tile_y=tile["tile_y"], zblock=tile["zblock"],
                               ctas_per_sm=tile["ctas_per_sm"], aligned=tile["aligned"],
                               skip_c=tile["skip_c"], tile_x=tile["tile_x"])
        from paper_1906_10811_b300 import binding as B

        def shot_sequence(n):
            """n shots back to back, as a seismic acquisition runs them: a shot's model upload
            overlaps the previous shot's steps (fd_set_model with host buffers),
            whose traces are read before the next shot's receivers replace them."""
            for i in range(n):
                se.set_model(m_h, damp_h)
                if i:
                    B.fd_read(se.ctx, None, rec_out if w["nrec"] else None)
                se.set_sources(src_h, wav_h)
                if w["nrec"]:
                    se.set_receivers(rc_h)
                se.reset()  # the shot starts from rest
                se.run(nt)
            B.fd_read(se.ctx, None, rec_out if w["nrec"] else None)

        shot_sequence(args.warmup)
        barrier()
        t0 = time.perf_counter()
        shot_sequence(args.steps)
        barrier()
        te = time.perf_counter() - t0
        se.close()
        te = reduce_max(te)
        e2e = {"value": round(whole_job_rate(npts * nt * args.steps, world, te) / 1e9, 3), "unit": "GPts/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_seconds)

    if rank == 0:
        line = {"metric": "GPts/s & % HBM roofline per stencil", "value": round(value, 3),
                "unit": "GPts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_of(args, w, kernel_name), tile=tile,
                               tile_choice=("autotuned over %d configurations" % tune_tried
                                            if tune_tried else
                                            "default" if args.tile == "default" else "given")),
                "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
        if world == 1 and args.workload == "acoustic256":
            run_extras(args, line, p)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def serving_result(args, rank=0, world=1):
    """Serve the seeded Poisson stream batched and one shot at a time, with the shots'
    m and damp in pageable host memory (the line's figures) and again in pinned host
    memory (``pinned_inputs``): the result line."""
    from paper_1906_10811_b300 import build
    from paper_1906_10811_b300.serve import (DeviceBackend, Server, ShotRequest, serve_sequential,
                                             summarize)
    build.build()
    stream = fdsynth.serving_stream(nshots=args.shots, seed=2 + rank, mean_gap_s=args.mean_gap)
    reqs = [ShotRequest(i, a, p) for i, a, p in stream]
    pts = sum(int(np.prod(p["shape"])) * p["nt"] for _, _, p in stream)
    # warm the library (module load, first graphs) on a small shot
    warm = fdsynth.serving_stream(nshots=2, seed=99, sizes2d=(64, 64), sizes3d=(32, 32),
                                  nt_range=(10, 10), nrec_range=(8, 8))
    serve_sequential([ShotRequest(i, 0.0, p) for i, _, p in warm])
    import torch
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    clocks = ClockSampler(gpu_id)
    be = DeviceBackend(8)
    srv = Server(be, hbm_budget=int(args.hbm_budget_gb * 2 ** 30), max_members=64,
                 ticks_per_round=args.ticks_per_round, work_cap=args.work_cap)
    batched = summarize(srv.serve(reqs))
    be.close()
    seq = summarize(serve_sequential(reqs))
    # the same stream with m and damp in pinned host memory (as a server that receives
    # requests into pinned buffers): their uploads no longer block the serving thread
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    preqs = [ShotRequest(r.id, r.arrival, dict(r.problem, m=pinned(r.problem["m"]),
                                               damp=pinned(r.problem["damp"]))) for r in reqs]
    be = DeviceBackend(8)
    srv = Server(be, hbm_budget=int(args.hbm_budget_gb * 2 ** 30), max_members=64,
                 ticks_per_round=args.ticks_per_round, work_cap=args.work_cap)
    pb = summarize(srv.serve(preqs))
    be.close()
    ps = summarize(serve_sequential(preqs))
    del preqs
    pinned_leg = {"serving": {k: round(v, 4) for k, v in pb.items()},
                  "sequential": {k: round(v, 4) for k, v in ps.items()},
                  "speedup_vs_sequential": round(pb["shots_per_s"] / ps["shots_per_s"], 3),
                  "p99_vs_sequential": round(pb["p99_s"] / ps["p99_s"], 3),
                  "host_bytes": int(sum(r.problem["m"].nbytes + r.problem["damp"].nbytes
                                        for r in reqs))}
    clk = clocks.stop()
    return {"metric": "served shots/s", "value": round(batched["shots_per_s"], 3),
            "unit": "shots/s", "n_gpus": world, "steps": args.shots, "warmup": 1,
            "ms_per_step": round(1e3 * batched["seconds"] / args.shots, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"poisson stream of {args.shots} acoustic shots, so 8",
                       "grids": "2-D 200^2-1000^2, 3-D 128^3-320^3", "nt": "300-1000",
                       "receivers": "128-512", "mean_gap_s": args.mean_gap,
                       "hbm_budget_gb": args.hbm_budget_gb, "grid_point_updates": pts,
                       "admission": "first come first served, tick work cap %d points" %
                                    args.work_cap,
                       "ticks_per_round": args.ticks_per_round},
            "serving": {k: round(v, 4) for k, v in batched.items()},
            "sequential": {k: round(v, 4) for k, v in seq.items()},
            "speedup_vs_sequential": round(batched["shots_per_s"] / seq["shots_per_s"], 3),
            "p99_vs_sequential": round(batched["p99_s"] / seq["p99_s"], 3),
            "gpts_per_s": round(pts / batched["seconds"] / 1e9, 2),
            "pinned_inputs": pinned_leg, "clocks": clk}


def run_serving(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    line = serving_result(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "fwi320":
        return run_fwi(args)
    if args.workload in ("diffusion512", "diffusion2d"):
        return run_diffusion(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
