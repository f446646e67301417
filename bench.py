#!/usr/bin/env python3
"""Benchmark of the reaction-diffusion stepper on GB300.

One bench step = one complete job of the 256^3 periodic Brusselator
(2 species, FP32 state, a=3, b=9, Du=2, Dv=16, dt=0.005): load the seeded
initial fields, then 10 000 forward-Euler steps through the fused kernel
(7-point Laplacian + reaction + Euler update, temporal blocking, CUDA-graph
replay).  Metric: GLUPS = cells x time steps / s / 1e9 (the paper's
Mpoints/s, scaled), aggregated over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-extras]
  python bench.py --serve [--serve-requests 500]      (serving workload)

Under torchrun each rank runs its own replica of the job (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1004_0480_gb300 import workloads as W  # noqa: E402

METRIC = "GLUPS (cell updates per second / 1e9), brusselator 256^3 FP32"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_FILE = os.path.join(ROOT, "profiles", "rd_step_brusselator_256.md")
WORKLOAD = "brusselator_256^3_periodic_10000_steps"
KERNEL_SOURCES = ["paper_1004_0480_gb300/csrc/rd_step_kernel.cuh",
                  "paper_1004_0480_gb300/csrc/rd_step1w_kernel.cuh",
                  "paper_1004_0480_gb300/csrc/rd_debug.cuh",
                  "paper_1004_0480_gb300/csrc/rd_k_brusselator.cu",
                  "paper_1004_0480_gb300/csrc/rd_internal.h"]


# ------------------------------------------------------------------ helpers
def dist_setup(n_gpus):
    """Rank layout from the torchrun environment; one process per GPU.
    NCCL where CUDA is present, else gloo (the CPU test of the N > 1 path)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The slowest rank's value (the job ends when every replica is done)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(cell_steps_per_rank, ws, elapsed_s):
    """Aggregate throughput: every rank's cell-steps over the slowest rank's
    time (weak scaling: each rank runs its own replica of the job)."""
    return cell_steps_per_rank * ws / elapsed_s / 1e9


def measured_peak():
    try:
        with open(PEAKS_FILE) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def kernel_sha():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(tsteps, tile_q, tile_y):
    """(DRAM bytes per launch, tuning they were taken at) from the committed
    ncu summary, if it was taken on the current kernel source at the same
    steps per launch and tile; else (None, None).  The register cap does not
    change what the kernel reads and writes; the z-chunk changes only how
    many halo planes are re-read (mostly from L2), so the tuning is reported
    beside the number instead of being required to match."""
    try:
        text = open(PROFILE_FILE).read()
    except OSError:
        return None, None
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    try:
        if fields.get("kernel_sha") != kernel_sha():
            return None, None
        if (int(fields["tsteps"]), int(fields["tile_q"]), int(fields["tile_y"])) != \
                (tsteps, tile_q, tile_y):
            return None, None
        tun = {k: int(fields[k]) for k in ("tsteps", "tile_q", "tile_y", "zchunk", "regcap")}
        return float(fields["dram_bytes_per_launch"]), tun
    except (KeyError, ValueError):
        return None, None


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                     hw=parts[5], hwt=parts[6], swt=parts[7], cap=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        smax = max(r["smax"] for r in rows)
        loaded = [r for r in rows if r["sm"] > 0.5 * smax] or rows
        reasons = set()
        for r in rows:
            if r["hw"].lower().startswith("active"):
                reasons.add("hw_slowdown")
            if r["hwt"].lower().startswith("active"):
                reasons.add("hw_thermal_slowdown")
            if r["swt"].lower().startswith("active"):
                reasons.add("sw_thermal_slowdown")
            if r["cap"].lower().startswith("active"):
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline
def host_cpu():
    """Model name and logical core count of the host running the oracle."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:      # Arm hosts: /proc/cpuinfo has no model name, lscpu does
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def oracle_sample(cfg, nsteps, fields=None):
    """Time the FP64 oracle (single thread) on ``nsteps`` steps of ``cfg``."""
    import oracle
    oracle.build()
    f = W.initial_fields(cfg) if fields is None else fields
    t0 = time.perf_counter()
    oracle.run(cfg, f, nsteps)
    dt = time.perf_counter() - t0
    return W.cell_count(cfg) * nsteps / dt / 1e9, dt


def reference_arm(args, ws, rank):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    if rank != 0:
        return 0
    cfg = W.cfg_brusselator_256()
    f = W.initial_fields(cfg)
    sample_steps = 1
    for _ in range(args.warmup):
        oracle_sample(cfg, sample_steps, f)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample(cfg, sample_steps, f)
        times.append(dt)
    tot = sum(times)
    glups = W.cell_count(cfg) * sample_steps * args.steps / tot / 1e9
    sample = (f"{sample_steps} forward-Euler step of the 256^3 Brusselator per bench step "
              f"(FP64 C oracle, single thread)")
    line = {
        "impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": W.cell_count(cfg), "species": 2,
                   "steps_per_job": cfg["steps"], "sample": sample},
        "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch

    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300.sim import Batch, Sim

    torch.cuda.set_device(local)
    if args.profile and args.profile_workload != "brusselator_256":
        return profile_other(args, Sim, torch)
    cfg = W.cfg_brusselator_256()
    steps_per_job = args.job_steps or cfg["steps"]
    cells = W.cell_count(cfg)
    f = W.initial_fields(cfg)
    stream = torch.cuda.Stream()
    sim = Sim(cfg, stream=stream)
    sim.set_fields(f)
    if args.tuning:
        sim.set_tuning(**parse_tuning(args.tuning))
        tun = sim.tuning()
    else:
        tun = sim.autotune()
    if args.profile:
        # a few single launches of the step kernel for an ncu capture
        for _ in range(args.profile):
            sim.step(tun["tsteps"])
        sim.sync()
        sim.close()
        return 0
    dev_ic = torch.from_numpy(f).cuda()
    host_ic = torch.from_numpy(f).pin_memory()
    host_out = torch.empty_like(host_ic).pin_memory()

    def job_device():
        for s in range(2):
            sim.set_field(s, dev_ic[s])
        sim.step(steps_per_job)

    for _ in range(args.warmup):
        job_device()
    sim.sync()

    # ---------------- timed region: device-resident inputs
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    step_kernel_ms = 0.0
    step_kernel_launches = 0
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        launches0 = sim.launches
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(args.steps):
            for s in range(2):
                sim.set_field(s, dev_ic[s])
            l0 = sim.launches
            ev[i][0].record(stream)
            sim.step(steps_per_job)
            ev[i][1].record(stream)
            step_kernel_launches += sim.launches - l0
        end.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        launches = sim.launches - launches0
    elapsed_ms = start.elapsed_time(end)
    step_kernel_ms = sum(a.elapsed_time(b) for a, b in ev)
    elapsed_ms = max_over_ranks(elapsed_ms, ws)
    clocks = clk.summary()
    total_cell_steps = cells * steps_per_job * args.steps * ws
    value = whole_job_glups(cells * steps_per_job * args.steps, ws, elapsed_ms * 1e-3)

    # roofline of the step kernel: 2 species x (read + write) x 4 B per cell-step
    T = tun["tsteps"]
    per_launch_ms = step_kernel_ms / step_kernel_launches
    bytes_per_launch = 16.0 * cells * T
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    traffic, traffic_tun = profiled_traffic(T, tun["tile_q"], tun["tile_y"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic, "traffic_tuning": traffic_tun,
                "peak_source": peak_src,
                "kernel": ("rd_step1_kernel<MBrusselator,float>" if T == 1
                           else f"rd_step_kernel<MBrusselator,float,{T}>"),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "launch_ms": per_launch_ms,
                "compulsory_frac": (16.0 * cells) / (per_launch_ms * 1e-3) / 1e9 / peak,
                # the same achieved bandwidth against the nominal 8 TB/s HBM3e figure
                "frac_of_nominal_8tbs": achieved / 8000.0}

    # ---------------- end to end through the C ABI with host buffers
    def job_host():
        for s in range(2):
            sim.set_field(s, host_ic[s])
        sim.step(steps_per_job)
        for s in range(2):
            sim.get_field(s, host_out[s])

    job_host()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        job_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    barrier(ws)
    e2e = {"value": total_cell_steps / e2e_s / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": int(host_ic.numel() * 4),
           "d2h_bytes_per_step": int(host_out.numel() * 4)}
    assert np.isfinite(host_out.numpy()).all()

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(args, Sim, Batch, torch)
        if args.bench_serve_requests > 0:
            extras["serving"] = serving_extra(args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        glups_cpu, dt = oracle_sample(cfg, args.cpu_steps, f)
        cpu = {"value": glups_cpu, "unit": "GLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_steps} steps of the 256^3 Brusselator, FP64 C oracle, "
                         f"single thread ({dt:.1f} s)", "host": host_cpu()}

    sim.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"brusselator_256^3_periodic_{steps_per_job}_steps", "cells": cells,
                   "species": 2, "steps_per_job": steps_per_job,
                   "l2": "state 2 x 128 MiB per level > 129 MB L2 (no flush needed)",
                   "tuning": tun, "parallelism": f"replicas x{ws}"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if extras:
        line["extras"] = extras
    print(json.dumps(line), flush=True)
    return 0


PROFILE_WORKLOADS = {
    # name: (problem, storage); the resident workload takes no --tuning
    "diffusion_64_resident": (lambda: W.cfg_diffusion_64(), "f32"),
    "air_512x512x64": (lambda: W.cfg_air_512(), "f32"),
    "ch_front_256": (lambda: W.ch_front(256), "f32"),
    "brusselator_256_19pt": (lambda: W.cfg_brusselator_256_19pt(), "f32"),
    "brusselator_256_bf16": (lambda: W.cfg_brusselator_256(), "bf16"),
    "ch_table1_192_19pt": (lambda: W.ch_table1(192), "f32"),
    "plume_144x144x384_19pt": (lambda: W.with_(W.plume(), stencil=19), "f32"),
}


def parse_tuning(text):
    """--tuning 'tsteps,tile_y,zchunk[,regcap[,tile_q]]' as rd_tuning fields."""
    vals = [int(x) for x in text.split(",")]
    t = dict(tsteps=vals[0], tile_y=vals[1], zchunk=vals[2],
             regcap=vals[3] if len(vals) > 3 else 0)
    if len(vals) > 4:
        t["tile_q"] = vals[4]
    return t


def profile_other(args, Sim, torch):
    """A few single launches of another workload's step kernel (for ncu):
    the problem with the given tuning, two warm-up steps, then ``--profile``
    single-step calls, no graph.  The resident workload instead runs its
    whole job (one launch) ``--profile`` times with the library's plan."""
    mk, storage = PROFILE_WORKLOADS[args.profile_workload]
    cfg = mk()
    if args.profile_workload.endswith("_resident"):
        with Sim(cfg, storage) as sim:
            sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
            sim.set_kernel("resident")
            for _ in range(args.profile):
                sim.step(cfg["steps"])
            sim.sync()
            print(json.dumps({"plan": sim.resident_plan()}), flush=True)
        return 0
    tun = parse_tuning(args.tuning)
    with Sim(cfg, storage) as sim:
        sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
        sim.set_tuning(graph=0, **tun)
        sim.step(2)
        for _ in range(args.profile):
            sim.step(tun["tsteps"])
        sim.sync()
    return 0


def _timed_steps(torch, sim, steps, reps=2):
    """Device time (CUDA events on the context's stream) of ``steps`` steps,
    best of ``reps``; the state keeps evolving, which does not change the
    work."""
    stream = torch.cuda.Stream()
    sim.set_stream(stream)
    sim.step(min(steps, 50))
    sim.sync()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return best


def _entry(cells, steps, seconds, bytes_per_cell_step, tuning=None, **kw):
    peak, _ = measured_peak()
    glups = cells * steps / seconds / 1e9
    d = {"glups": glups, "cells": cells, "steps": steps,
         "bytes_per_cell_step": bytes_per_cell_step,
         "roofline_frac": glups * bytes_per_cell_step / peak}
    if tuning is not None:
        d["tuning"] = tuning
    d.update(kw)
    return d


def run_extras(args, Sim, Batch, torch):
    """The other workloads: GLUPS and fraction of the measured HBM peak
    (algorithmic bytes 2 x species x bytes per value per cell-step)."""
    out = {}
    # Brusselator 256^3 with BF16 storage (8 B per cell-step)
    cfg = W.cfg_brusselator_256()
    with Sim(cfg, storage="bf16") as sim:
        sim.set_fields(W.initial_fields(cfg))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 2000)
        out["brusselator_256_bf16"] = _entry(W.cell_count(cfg), 2000, t, 8, tun)
    # the same problem with the paper's 19-point Laplacian, eqs. (3)-(4)
    # (FP32, the same 16 B per cell-step)
    cfg = W.cfg_brusselator_256_19pt()
    with Sim(cfg) as sim:
        sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 2000)
        out["brusselator_256_19pt"] = _entry(W.cell_count(cfg), 2000, t, 16, tun)
    # the Turing system of Table 1 with its parameters on the paper's 192^3
    # grid and its 19-point stencil (2 levels x 2 species x 28 MiB: the
    # working set fits the 129 MB L2), and on 256^3 (beyond L2)
    for n in (192, 256):
        tcfg = W.turing(n, stencil=19)
        with Sim(tcfg) as sim:
            sim.set_fields(W.initial_fields_torch(tcfg, "cuda"))
            tun = sim.autotune()
            t = _timed_steps(torch, sim, 2000)
            out[f"turing_{n}_19pt"] = _entry(W.cell_count(tcfg), 2000, t, 16, tun)
    # the Cahn-Hilliard row of Table 1 with its parameters, 19-point stencil
    # and the paper's 192^3 grid: two launches per step (mu, then the
    # update), 36 B per cell-step moved by the two launches against the 24 B
    # algorithmic minimum the fraction is stated at
    ccfg = W.ch_table1(192)
    with Sim(ccfg) as sim:
        sim.set_fields(W.initial_fields_torch(ccfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 1000)
        out["ch_table1_192_19pt"] = _entry(W.cell_count(ccfg), 1000, t, 24, tun,
                                           launches_per_step=2, moved_bytes_per_cell_step=36)
    # the plume of Table 1 (row 4) on its 144 x 144 x 384 grid with the
    # 19-point stencil: upwind along three axes, u_z = 5 sin(t / 500 s) read
    # from the device step counter (1 species, 8 B per cell-step)
    pcfg = W.with_(W.plume(), stencil=19)
    with Sim(pcfg) as sim:
        sim.set_fields(W.initial_fields_torch(pcfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 2000)
        out["plume_144x144x384_19pt"] = _entry(W.cell_count(pcfg), 2000, t, 8, tun)
    # the paper's own kernel designs on the same problem (ablation baselines:
    # Shared method and Moving Tiles, Section 4.1, Tables 4-5)
    for kern in ("shared", "tiles"):
        with Sim(cfg) as sim:
            sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
            sim.set_kernel(kern)
            t = _timed_steps(torch, sim, 400)
            out[f"brusselator_256_19pt_{kern}"] = _entry(W.cell_count(cfg), 400, t, 16,
                                                         kernel=kern)
    # inert diffusion 64^3, 100 steps (L2-resident: launch-bound, not HBM)
    cfg = W.cfg_diffusion_64()
    with Sim(cfg) as sim:
        sim.set_fields(W.initial_fields(cfg))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, cfg["steps"], reps=5)
        out["diffusion_64"] = _entry(W.cell_count(cfg), cfg["steps"], t, 8, tun,
                                     note="1 MiB per level: L2-resident, launch-bound")
    # the same run with the resident kernel: one cooperative launch for the
    # 100 steps, a grid-wide barrier between steps (same bits as above)
    with Sim(cfg) as sim:
        sim.set_fields(W.initial_fields(cfg))
        sim.set_kernel("resident")
        t = _timed_steps(torch, sim, cfg["steps"], reps=5)
        out["diffusion_64_resident"] = _entry(W.cell_count(cfg), cfg["steps"], t, 8,
                                              kernel="resident", plan=sim.resident_plan(),
                                              note="one launch for the 100 steps, K steps "
                                                   "per grid barrier, state in L2")
    # the same kinetics at 512^3 (1 GiB per level) for the HBM roofline
    cfg = W.diffusion_blob(512, steps=400, dt=0.1)
    with Sim(cfg) as sim:
        sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 400)
        out["diffusion_512"] = _entry(W.cell_count(cfg), 400, t, 8, tun)
    # the front model (Cahn-Hilliard) on one 256^3 instance (24 B per cell-step)
    fcfg = W.ch_front(256)
    with Sim(fcfg) as sim:
        sim.set_fields(W.initial_fields_torch(fcfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 1000)
        out["ch_front_256"] = _entry(W.cell_count(fcfg), 1000, t, 24, tun)
    # air 512 x 512 x 64, 3 species (24 B per cell-step)
    cfg = W.cfg_air_512()
    with Sim(cfg) as sim:
        sim.set_fields(W.initial_fields_torch(cfg, "cuda"))
        tun = sim.autotune()
        t = _timed_steps(torch, sim, 1000)
        out["air_512x512x64"] = _entry(W.cell_count(cfg), 1000, t, 24, tun)
    # 32 uneven front instances (3 species, 24 B per cell-step), full 2000
    # steps: one batched launch sequence vs the plain stepper
    cfgs = W.cfg_ch_front_batch(steps=args.batch_steps)
    cells_b = sum(W.cell_count(c) for c in cfgs)
    sims = [Sim(c) for c in cfgs]
    for c, sm in zip(cfgs, sims):
        sm.set_fields(W.initial_fields_torch(c, "cuda"))
    stream = torch.cuda.Stream()
    b = Batch("ch_front", stream=stream)
    # 12-row tiles and 48-plane chunks (measured best for these members with
    # work items pulled from the batch's counter: 129 GLUPS against 128 for
    # 32-plane chunks, 125 for 10-row and 116 for 16-row tiles)
    btun = dict(tsteps=1, tile_q=16, tile_y=12, zchunk=48, graph=1)
    b.set_tuning(**btun)
    for sm in sims:
        b.add(sm)
    b.step(20)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.batch_steps)
    e1.record(stream)
    e1.synchronize()
    bt = e0.elapsed_time(e1) * 1e-3
    for sm in sims:
        b.remove(sm)
    b.close()
    # plain stepper: the fused kernel at T=1, one launch per instance and
    # step, no graph, instances serialised in arrival order on one stream
    common = torch.cuda.Stream()
    for sm in sims:
        sm.set_tuning(tsteps=1, graph=0)
        sm.set_stream(common)
    torch.cuda.synchronize()
    e0.record(common)
    for sm in sims:
        sm.step(args.batch_steps)
    e1.record(common)
    e1.synchronize()
    pt = e0.elapsed_time(e1) * 1e-3
    for sm in sims:
        sm.close()
    out["ch_front_batch_32"] = {
        "instances": len(cfgs),
        "batched": _entry(cells_b, args.batch_steps, bt, 24, btun),
        "plain": _entry(cells_b, args.batch_steps, pt, 24, dict(tsteps=1, graph=0)),
        "speedup": pt / bt}
    return out


def serving_setup(args, SV, count):
    """The seeded request mix, every family warmed up once (first use of a
    kernel and of the device field generator costs seconds of one-time
    loading per process), and the plain stepper's capacity measured on the
    first few requests of the mix (cell-steps per second, each request's
    context creation and upload included)."""
    import torch
    specs = W.serving_requests(count=count, rate_per_s=1.0, seed=4)
    reqs = SV.requests_from_workload(specs)
    mean_work = float(np.mean([r.cells * r.steps for r in reqs]))
    warm = [SV.Request(-1 - i, 0.0, mk(16, steps=4))
            for i, mk in enumerate((W.diffusion_blob, W.brusselator, W.ch_front))]
    eng = SV.CudaEngine()
    for r in warm:
        eng.run_alone(r, False)
    server = SV.Server(SV.CudaEngine(), budget_bytes=args.serve_budget_gb * 1e9,
                       quantum=args.serve_quantum, run_cells=args.serve_run_cells)
    server.run(warm)
    server.engine.shutdown()
    torch.cuda.synchronize()
    probe = reqs[: max(3, min(8, len(reqs)))]
    t0 = time.perf_counter()
    for r in probe:
        eng.run_alone(r, False)
    torch.cuda.synchronize()
    cap = sum(r.cells * r.steps for r in probe) / (time.perf_counter() - t0)
    return reqs, cap, mean_work


def serving_pack(st):
    return {"p50_s": st.p50, "p99_s": st.p99, "mean_s": st.mean, "glups": st.glups,
            "makespan_s": st.makespan, "max_active": st.max_active,
            "max_running": st.max_running, "max_device_bytes": st.max_bytes,
            "gpu_launches": st.launches}


def serving_at_load(args, SV, reqs, cap, mean_work, load, progress=None):
    """Both servers on the same Poisson stream at ``load`` x the plain
    capacity: (continuous batching stats, plain stats, arrival rate)."""
    rate = load * cap / mean_work
    rr = SV.with_rate(reqs, rate, seed=4)
    server = SV.Server(SV.CudaEngine(), budget_bytes=args.serve_budget_gb * 1e9,
                       quantum=args.serve_quantum, run_cells=args.serve_run_cells,
                       progress=progress)
    _, st_b = server.run(rr)
    server.engine.shutdown()
    _, st_p = SV.serve_plain(SV.CudaEngine(), rr, progress=progress)
    return st_b, st_p, rate


def serving_extra(args):
    """The reduced serving run of the default bench line: the first
    ``--bench-serve-requests`` requests of the mix at ``--serve-load``."""
    from paper_1004_0480_gb300 import serving as SV
    reqs, cap, mean_work = serving_setup(args, SV, args.bench_serve_requests)
    st_b, st_p, rate = serving_at_load(args, SV, reqs, cap, mean_work, args.serve_load)
    return {"requests": len(reqs), "offered_load": args.serve_load,
            "arrival_rate_per_s": rate, "plain_capacity_glups": cap / 1e9,
            "continuous_batching": serving_pack(st_b), "plain": serving_pack(st_p),
            "p99_speedup": st_p.p99 / st_b.p99 if st_b.p99 > 0 else None,
            "p50_speedup": st_p.p50 / st_b.p50 if st_b.p50 > 0 else None}


def run_serving(args):
    """Serving workload: seeded Poisson stream of mixed requests, served by
    continuous batching and by the plain one-request-at-a-time stepper."""
    import torch

    from paper_1004_0480_gb300 import build as B
    B.build()
    from paper_1004_0480_gb300 import serving as SV

    torch.cuda.set_device(0)
    reqs, cap, mean_work = serving_setup(args, SV, args.serve_requests)
    if args.serve_loads:
        return serving_sweep(args, SV, reqs, cap, mean_work)
    rate = args.serve_load * cap / mean_work
    if args.serve_progress:
        print(f"serve plain capacity {cap / 1e9:.1f} GLUPS, arrival rate {rate:.3f}/s",
              file=sys.stderr, flush=True)
    last = [0.0]

    def progress(t, n_adm, n_run, n_done):
        # one line every 10 s on stderr, with --serve-progress
        if args.serve_progress and (t < last[0] or t - last[0] >= 10.0):
            last[0] = t
            print(f"serve t={t:.1f}s admitted={n_adm} running={n_run} done={n_done}",
                  file=sys.stderr, flush=True)
    st_b, st_p, rate = serving_at_load(args, SV, reqs, cap, mean_work, args.serve_load,
                                       progress)
    rr = SV.with_rate(reqs, rate, seed=4)
    # capacity: the first requests of the stream all arriving at once
    sat = [SV.Request(r.id, 0.0, r.cfg) for r in rr[: args.serve_sat_requests]]
    server = SV.Server(SV.CudaEngine(), budget_bytes=args.serve_budget_gb * 1e9,
                       quantum=args.serve_quantum, run_cells=args.serve_run_cells,
                       progress=progress)
    _, sat_b = server.run(sat)
    server.engine.shutdown()
    _, sat_p = SV.serve_plain(SV.CudaEngine(), sat, progress=progress)
    line = {
        "metric": "serving latency p50/p99 (s) and aggregate GLUPS", "unit": "s",
        "requests": len(reqs), "arrival_rate_per_s": rate, "offered_load": args.serve_load,
        "plain_capacity_glups": cap / 1e9, "budget_gb": args.serve_budget_gb,
        "quantum_steps": args.serve_quantum, "run_cells": args.serve_run_cells,
        "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals, diffusion/brusselator/ch_front "
                               "kinetics, edges {32..384}^3, 100..5000 steps", "seed": 4},
        "continuous_batching": serving_pack(st_b), "plain": serving_pack(st_p),
        "p99_speedup": st_p.p99 / st_b.p99 if st_b.p99 > 0 else None,
        "saturated": {"requests": len(sat), "continuous_batching": serving_pack(sat_b),
                      "plain": serving_pack(sat_p),
                      "glups_speedup": sat_b.glups / sat_p.glups if sat_p.glups > 0 else None},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_sweep(args, SV, reqs, cap, mean_work):
    """Both servers at each offered load of --serve-loads (fraction of the
    plain stepper's measured capacity); one JSON line."""
    rows = []
    for load in (float(x) for x in args.serve_loads.split(",")):
        st_b, st_p, rate = serving_at_load(args, SV, reqs, cap, mean_work, load)
        rows.append({"offered_load": load, "arrival_rate_per_s": rate,
                     "continuous_batching": {"p50_s": st_b.p50, "p99_s": st_b.p99,
                                             "mean_s": st_b.mean, "glups": st_b.glups},
                     "plain": {"p50_s": st_p.p50, "p99_s": st_p.p99, "mean_s": st_p.mean,
                               "glups": st_p.glups}})
    print(json.dumps({"metric": "serving latency p50/p99 (s) and aggregate GLUPS vs offered load",
                      "unit": "s", "requests": len(reqs), "plain_capacity_glups": cap / 1e9,
                      "run_cells": args.serve_run_cells, "quantum_steps": args.serve_quantum,
                      "data": "synthetic", "sweep": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--job-steps", type=int, default=0,
                    help="time steps per job (default: the workload's 10 000)")
    ap.add_argument("--tuning", default="",
                    help="fixed tuning 'tsteps,tile_y,zchunk[,regcap[,tile_q]]' instead of the "
                         "autotuner")
    ap.add_argument("--profile", type=int, default=0,
                    help="only run this many single step-kernel launches (for ncu)")
    ap.add_argument("--profile-workload", default="brusselator_256",
                    choices=["brusselator_256", *PROFILE_WORKLOADS],
                    help="workload of --profile (the others need --tuning)")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload instead of the step benchmark")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="offered load as a fraction of the plain stepper's capacity")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-quantum", type=int, default=250)
    ap.add_argument("--serve-loads", default="",
                    help="comma-separated offered loads: run both servers at each instead")
    ap.add_argument("--serve-progress", action="store_true",
                    help="report the serving loop's progress on stderr every 10 s")
    ap.add_argument("--serve-run-cells", type=float, default=48e6,
                    help="cells the running requests hold together (inf: all admitted run)")
    ap.add_argument("--serve-sat-requests", type=int, default=100,
                    help="requests of the saturated (all arrive at once) capacity run")
    ap.add_argument("--bench-serve-requests", type=int, default=100,
                    help="requests of the reduced serving run in the default line's "
                         "extras (0: none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.serve:
        return run_serving(args)
    ws, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        rc = reference_arm(args, ws, rank)
    else:
        rc = run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
