#!/usr/bin/env python
"""Throughput of the fully discrete third-order Active Flux step on GB300.

One benchmark step = one time step of the whole hot path (ghost fill, cell
prep, point values at t^{n+1/2} and t^{n+1} with the correction term and the
bound-preserving limiter, Simpson fluxes and the finite-volume update, plus
the max-speed reduction that sets dt) over the 8192 x 8192 isentropic-vortex
grid on the periodic box [0,10]^2, centre and strength drawn from seed 2508.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (launched by torch.distributed.run)
every rank advances its own independent grid (replicas, weak scaling).  The
reference arm (--impl reference) times the FP64 CPU oracle on the host cores
on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell updates/s (FP32 plain vs MLP-surrogate+fallback) at stated L1 error vs FP64 oracle"
UNIT = "cell updates/s"
SEED = 2508
# FP32 operations of the point-value stage per cell update, counted from the
# kernel source (add, sub, mul = 1, fma = 2; sqrt, div and transcendental
# calls not counted) for this workload's background state (u = v = 1,
# c = 1.18: both grid lines cross every Mach circle, the node lies outside
# it, so X and Y do not meet): a vertex (3 cells' circle coefficients, two
# half-circle tables: 1057) and two edge midpoints (2 cells, one half-circle
# table: 670 each) at two time levels, plus the correction term, the
# linearisation state and the fused cell prep (809): 5.6 k.  Vortex-core
# vertices, whose circles also need the quarter arc, do 472 more.  The FP32
# operations the kernel executes on this workload (ncu: fadd + fmul + 2 ffma)
# are 5.55 k a cell update, 1% under the count (the compiler folds some of
# what it counts): the achieved figure takes 5.5 k, below both.
PV_FLOP_PER_CELL = 5500
# algorithmic HBM bytes of the flux/update kernel per cell: 3 levels x 3 node
# arrays read (144 B), averages hi/lo read and written (64 B)
FLUX_BYTES_PER_CELL = 208
# DRAM bytes (read + write) per cell update of the point-value and flux
# kernels from one ncu capture (2048^2 case, scaled per cell: every array is
# read or written once per launch), valid only for the kernel sources they
# were taken on (sha256 of the kernel's file and of the shared inline device
# code; af_kernels.h, which declares every kernel's launcher, is left out);
# otherwise reported as null
_KSRC = "paper_2508_06273_gb300/csrc/"
_SHARED = {_KSRC + "af_common.cuh": "093115c23be2e775d5d20529727a61310b8bf8c4402d8e1bf8500c33560da0aa"}
PV_TRAFFIC = {"bytes_per_cell": 150.8, "profile": "profiles/dram_pointvalue_flux_vortex2048.md",
              "sha256": dict(_SHARED, **{_KSRC + "af_pointvalue.cu":
                                         "5dd8c49de21a3549206c6886e2b4104ff62e4ac106776ebf97ec4a8a3fad0121"})}
FLUX_TRAFFIC = {"bytes_per_cell": 206.6, "profile": "profiles/dram_pointvalue_flux_vortex2048.md",
                "sha256": dict(_SHARED, **{_KSRC + "af_flux.cu":
                                           "164c4a83daa94e5a5764bed37528724938990583775d6600124f0663476ded73"})}


def measured_traffic(spec, cells):
    """Per-launch DRAM bytes from a capture, or None if the source changed since."""
    import hashlib

    for rel, digest in spec["sha256"].items():
        try:
            if hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest() != digest:
                return None
        except OSError:
            return None
    return spec["bytes_per_cell"] * cells


# ------------------------------------------------------------ distributed
def dist_setup(backend=None):
    """(rank, world, local_rank); initialises torch.distributed when WORLD_SIZE > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def reduce_max(x, world, device=None):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(cells_per_rank, steps, world, max_seconds):
    """Whole-job cell updates per second: all ranks' work over the slowest rank's time."""
    return cells_per_rank * steps * world / max_seconds


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu is not None:
            cmd += ["-i", str(self.gpu)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ helpers
def workload(n, rank=0):
    from paper_2508_06273_gb300 import workloads as W

    return W.shu_vortex_seeded(n, seed=SEED + rank)


def workload_name(n):
    return (f"isentropic vortex, periodic [0,10]^2, {n}x{n} cells, centre and strength "
            f"in [3,6] from seed {SEED}, CFL 0.3, one time step per bench step")


class OracleWindow:
    """FP64 oracle on a window of the workload around the vortex (outflow
    ghosts at its edge), on all host cores unless threads is given; one call
    = one time step (max-speed reduction + step)."""

    def __init__(self, n, window=128, threads=None):
        import numpy as np

        import oracle
        from paper_2508_06273_gb300 import workloads as W

        prob = workload(n)
        xc, yc = np.random.default_rng(SEED).uniform(3.0, 6.0, size=2)
        i0 = max(0, min(n - window, int(xc / prob.dx) - window // 2))
        j0 = max(0, min(n - window, int(yc / prob.dy) - window // 2))
        self.sub = W.subproblem(prob, i0, j0, window, window)
        self.cells = window * window
        self.window = window
        self.o = oracle.Oracle(self.sub.nx, self.sub.ny, self.sub.dx, self.sub.dy, self.sub.gamma,
                               self.sub.bc)
        self.threads = threads or len(os.sched_getaffinity(0))
        self.o.set_option(oracle.OPT_THREADS, self.threads)
        self.o.set_state(*W.to_f32(W.discretise(self.sub)))

    def step(self):
        self.o.step(self.sub.cfl * self.sub.dx / self.o.max_speed())

    def describe(self, n, steps):
        return (f"FP64 oracle on a {self.window}x{self.window}-cell window of the {n}^2 workload "
                f"around the vortex, {steps} steps (max-speed reduction + step), "
                f"{self.threads} OpenMP thread{'s' if self.threads > 1 else ''}")


def accuracy_leg(torch, af, W, n, steps=4, window=128):
    """Relative L1 of the GPU state of the bench workload against the FP64
    oracle on a window around the vortex (same initial FP32 data, same fixed
    dt), over the window's interior that the window's outflow edges cannot
    reach in ``steps`` steps; and the L1 error of rho against the exact
    vortex there."""
    import numpy as np

    prob = workload(n)
    s = af.Solver(n, n, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*W.discretise_torch(prob, "cuda"))
    win = OracleWindow(n, window)
    dt = prob.cfl * prob.dx / s.max_speed()
    for _ in range(steps):
        s.step(dt)
        win.o.step(dt)
    sub = win.sub
    i0, j0 = int(round((sub.x0 - prob.x0) / prob.dx)), int(round((sub.y0 - prob.y0) / prob.dy))
    m = 2 * steps + 2
    gpu = [a.double().cpu().numpy() for a in s.get_state()]
    s.close()
    ora = win.o.get_state()
    worst = 0.0
    for a, b in zip(gpu, ora):
        ga = a[:, j0 + m:j0 + window - m, i0 + m:i0 + window - m]
        ob = b[:, m:window - m, m:window - m]
        for v in range(4):
            scale = np.abs(ob[v]).sum() if v in (0, 3) else (np.abs(ob[1]) + np.abs(ob[2]) + 1.0).sum()
            worst = max(worst, float(np.abs(ga[v] - ob[v]).sum() / scale))
    ex = W.discretise(sub, sub.exact(steps * dt))[0][0][m:window - m, m:window - m]
    rho = gpu[0][0][j0 + m:j0 + window - m, i0 + m:i0 + window - m]
    return {"rel_l1_vs_oracle": worst, "l1_rho_vs_exact": float(np.abs(rho - ex).mean()),
            "l1_rho_oracle_vs_exact": float(np.abs(ora[0][0][m:window - m, m:window - m] - ex).mean()),
            "sample": f"{steps} steps of fixed dt on the {n}^2 grid; a {window}^2-cell window around the vortex "
                      f"in the oracle; compared on its {window - 2 * m}^2 interior; all arrays, worst variable"}


def cpu_sample(n, min_seconds=10.0, window=128, max_steps=200, threads=None):
    """(cell updates/s, threads, description, seconds) of the oracle window
    (on all host cores unless threads is given)."""
    w = OracleWindow(n, window, threads)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        w.step()
        steps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    el = time.perf_counter() - t0
    return w.cells * steps / el, w.threads, w.describe(n, steps), el


def fp32_peak_tflops(sm_count, mhz):
    """FP32 (non-tensor) peak: SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# ------------------------------------------------------------ arms
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_06273_gb300 import af
    from paper_2508_06273_gb300 import workloads as W

    n = args.grid
    prob = workload(n, rank)
    cells = n * n
    dev = W.discretise_torch(prob, "cuda")
    s = af.Solver(n, n, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*dev)
    pinned = None
    if args.e2e_steps > 0:
        pinned = [torch.empty(a.shape, dtype=torch.float32, pin_memory=True) for a in dev]
        for p, a in zip(pinned, dev):
            p.copy_(a)
    del dev
    torch.cuda.empty_cache()

    def one_step():
        dt = prob.cfl * prob.dx / s.max_speed()
        s.step(dt)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if s.status() != 0:
        raise SystemExit("warm-up steps raised device status bits")
    # point-value tile height: time two steps at each height, keep the fastest
    # (the result does not depend on it)
    tune = {}
    dt_t = prob.cfl * prob.dx / s.max_speed()
    for th in (4, 8, 16):
        s.set_option("tile_h", th)
        s.step(dt_t)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        s.step(dt_t)
        s.step(dt_t)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        tune[th] = e0.elapsed_time(e1) / 2
    tile_h = min(tune, key=tune.get)
    s.set_option("tile_h", tile_h)
    s.set_option("profile", 1)
    s.profile(reset=True)
    clocks = ClockSampler(local).start() if rank == 0 else None
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        one_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    status = s.status()
    stage_ms, launches = s.profile()
    s.set_option("profile", 0)
    max_s = reduce_max(ms / 1e3, world, device="cuda")
    value = aggregate_value(cells, args.steps, world, max_s)

    # end to end through the C ABI with host buffers: every step uploads its
    # inputs from pinned memory, steps (dt from the uploaded state's max
    # speed) and downloads the whole result into pinned memory, through the
    # asynchronous host calls, so that the download of one step overlaps the
    # upload of the next; the clock stops when the last download has landed
    e2e = None
    if pinned is not None:
        h2d = sum(p.numel() * 4 for p in pinned)
        outs = [torch.empty(p.shape, dtype=torch.float32, pin_memory=True).numpy() for p in pinned]
        host_in = [p.numpy() for p in pinned]
        s.set_state_host_async(*host_in)
        one_step()
        s.get_state_host_async(outs)
        s.host_sync()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            s.set_state_host_async(*host_in)
            one_step()
            s.get_state_host_async(outs)
        s.host_sync()
        torch.cuda.synchronize()
        el = reduce_max(time.perf_counter() - t0, world, device="cuda")
        e2e = {"value": aggregate_value(cells, args.e2e_steps, world, el), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d, "steps": args.e2e_steps,
               "transfers": "asynchronous host calls: upload k+1 overlaps download k and step k"}
    s.close()

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    pv_ms = stage_ms["pointvalue"] / args.steps
    pv_tflops = PV_FLOP_PER_CELL * cells / (pv_ms / 1e3) / 1e12
    peak = fp32_peak_tflops(sms, max_mhz)
    flux_ms = stage_ms["flux"] / args.steps
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        hbm_src = "measured"
    except (OSError, KeyError, ValueError):
        hbm, hbm_src = 6800.0, "fallback"
    flux_gbs = FLUX_BYTES_PER_CELL * cells / (flux_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(n), "cells": cells, "grid": [n, n],
                   "method": "Alg. 1 step, averaged linearisation, correction on, Alg. 3 limiter on",
                   "l2": "inputs larger than L2 (about 15 GB of state per grid)",
                   "tile_h": tile_h, "tile_ms_per_step": tune,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "node_updates_per_s": 3 * value,
        "status": status,
        "roofline": {"bound": "alu", "kernel": "point-value stage (1 launch: fused cell prep, vertices and edge midpoints)",
                     "achieved": pv_tflops, "peak": peak, "unit": "TFLOP/s", "frac": pv_tflops / peak,
                     "traffic": measured_traffic(PV_TRAFFIC, cells), "traffic_unit": "B per launch",
                     "traffic_source": PV_TRAFFIC["profile"], "flop_per_cell": PV_FLOP_PER_CELL,
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz (max clock)",
                     "frac_at_median_clock": (pv_tflops / fp32_peak_tflops(sms, clk["sm_mhz"])
                                              if clk else None),
                     "ms_per_launch": pv_ms},
        "roofline_flux": {"bound": "hbm", "kernel": "Simpson flux + compensated (double-word FP32) update", "achieved": flux_gbs,
                          "peak": hbm, "unit": "GB/s", "frac": flux_gbs / hbm, "peak_source": hbm_src,
                          "traffic": measured_traffic(FLUX_TRAFFIC, cells), "traffic_unit": "B per launch",
                          "traffic_source": FLUX_TRAFFIC["profile"],
                          "bytes_per_cell": FLUX_BYTES_PER_CELL, "ms_per_launch": flux_ms},
        "roofline_step": {
            "note": "whole step: point-value flops by the hand count, flux arithmetic not counted; DRAM bytes "
                    "of both kernels from their captures (the split design; 160 B would be a fused ideal)",
            "tflops": PV_FLOP_PER_CELL * cells / (max_s / args.steps) / 1e12,
            "frac_fp32": PV_FLOP_PER_CELL * cells / (max_s / args.steps) / 1e12 / peak,
            "bytes_per_cell": PV_TRAFFIC["bytes_per_cell"] + FLUX_TRAFFIC["bytes_per_cell"],
            "gbs": (PV_TRAFFIC["bytes_per_cell"] + FLUX_TRAFFIC["bytes_per_cell"]) * cells / (max_s / args.steps) / 1e9,
        },
        "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "gpu_launches": int(sum(launches.values())),
        "clocks": clk,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu:
        line["accuracy"] = accuracy_leg(torch, af, W, n)
    if world == 1 and args.batch_steps > 0:
        line["batch"] = run_batch_leg(args, torch, af, W)
    refs = None
    if world == 1 and not args.no_cpu and (args.surrogate or args.convergence):
        refs = oracle_references(af, W, args)
    if world == 1 and not args.no_cpu and args.convergence:
        line["convergence"] = convergence_leg(torch, af, W, refs)
    if world == 1 and args.surrogate:
        line["surrogate"] = run_surrogate_leg(args, torch, af, W, refs)
    if world == 1 and not args.no_cpu:
        v, threads, desc, _ = cpu_sample(n, min_seconds=args.cpu_seconds)
        v1, _, desc1, _ = cpu_sample(n, min_seconds=0.5 * args.cpu_seconds, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
                                "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": desc1}}
    print(json.dumps(line), flush=True)


def _oracle_run(af, W, prob, t_end, max_steps=1_000_000):
    """FP64 oracle from the FP32-rounded initial data of ``prob`` to t_end,
    dt = cfl h / (max speed) each step (the last step clipped), on all host
    cores.  Returns (state, dts, seconds)."""
    import oracle

    o = oracle.Oracle(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc)
    o.set_option(oracle.OPT_THREADS, len(os.sched_getaffinity(0)))
    for k, v in prob.options.items():
        o.set_option(af.OPT[k], v)
    o.set_state(*W.to_f32(W.discretise(prob)))
    t, dts, t0 = 0.0, [], time.perf_counter()
    while t < t_end * (1 - 1e-12) and len(dts) < max_steps:
        speed = o.max_speed()
        if not speed > 0.0 or speed == float("inf"):
            raise RuntimeError(f"oracle: wave speed {speed} at step {len(dts)}, t = {t:.6g}")
        dt = min(prob.cfl * min(prob.dx, prob.dy) / speed, t_end - t)
        o.step(dt)
        dts.append(dt)
        t += dt
    return o.get_state(), dts, time.perf_counter() - t0


def _gpu_replay(torch, af, W, prob, dts, nets=None, surr_opts=None):
    """GPU run of ``prob`` from the same FP32 initial data with the given dt
    sequence (plain, or the surrogate with exact fallback and the options
    surr_opts when nets are given).  Returns (state as float64 arrays,
    status, fallback fraction)."""
    import numpy as np

    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options=prob.options)
    s.set_state(*[torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
                  for a in W.to_f32(W.discretise(prob))])
    if nets:
        s.set_surrogate(nets[0], nets[1])
        for k, v in (surr_opts or {}).items():
            s.set_option(k, v)
    status = 0
    for dt in dts:
        s.step(dt)
    status |= s.status()
    frac = None
    if nets:
        n_net, n_fall = s.surrogate_stats()
        frac = n_fall / max(1, n_net + n_fall)
    out = [a.double().cpu().numpy() for a in s.get_state()]
    s.close()
    return out, status, frac


def _rel_l1(a_state, b_state):
    """max over the four arrays and variables of sum|a - b| / scale, the
    scale sum|b| for rho and p (E), sum(|u| + |v| + 1) for the velocities
    (momenta): the relative L1 the accuracy figures use."""
    import numpy as np

    worst = 0.0
    for a, b in zip(a_state, b_state):
        for v in range(4):
            scale = np.abs(b[v]).sum() if v in (0, 3) else (np.abs(b[1]) + np.abs(b[2]) + 1.0).sum()
            worst = max(worst, float(np.abs(a[v] - b[v]).sum() / scale))
    return worst


def _vortex_l1_vs_exact(W, prob, rho, t, radius=2.5):
    """mean |rho - rho_exact| over the cell averages: the whole box, and the
    cells within ``radius`` of the moving vortex centre (periodic distance)."""
    import numpy as np

    ex = W.discretise(prob, prob.exact(t))[0][0]
    err = np.abs(rho - ex)
    xc = prob.x0 + prob.dx * (np.arange(prob.nx) + 0.5)
    yc = prob.y0 + prob.dy * (np.arange(prob.ny) + 0.5)
    cx, cy = prob.vortex_centre(t)
    L = prob.lx
    dx = (xc[None, :] - cx + 0.5 * L) % L - 0.5 * L
    dy = (yc[:, None] - cy + 0.5 * L) % L - 0.5 * L
    near = dx * dx + dy * dy <= radius * radius
    return float(err.mean()), float(err[near].mean())


def oracle_references(af, W, args):
    """FP64 oracle runs the accuracy legs compare with (host cores, FP32
    initial data): the seeded vortex at 128^2 and 256^2 to t = 2 (K2), the
    four-quadrant problem of seed 6 at 256^2 to the Riemann leg's final time."""
    refs = {}
    for n in (128, 256):
        prob = W.shu_vortex_seeded(n, t_end=2.0, vel=W.STABLE_VELOCITY)
        refs[f"vortex{n}"] = (prob,) + _oracle_run(af, W, prob, 2.0)
    prob = W.four_quadrant(256, seed=6)
    refs["riemann256"] = (prob,) + _oracle_run(af, W, prob, args.riemann_t)
    return refs


def convergence_leg(torch, af, W, refs, seg_steps=400):
    """Isentropic-vortex sweep (seed 2508 law): 128^2 and 256^2 to t = 2
    against the FP64 oracle (same dt sequence) and the exact solution; 512^2
    and 2048^2 to t = 2 on the GPU against the exact solution, the 2048^2 run
    with its conserved totals every step; 8192^2 for ``seg_steps`` steps of
    fixed dt."""
    import numpy as np

    out = {}
    for n in (128, 256):
        prob, ora, dts, osec = refs[f"vortex{n}"]
        gpu, status, _ = _gpu_replay(torch, af, W, prob, dts)
        t = float(sum(dts))
        g_all, g_near = _vortex_l1_vs_exact(W, prob, gpu[0][0], t)
        o_all, o_near = _vortex_l1_vs_exact(W, prob, ora[0][0], t)
        out[f"{n}^2"] = {"t": t, "steps": len(dts), "rel_l1_vs_oracle": _rel_l1(gpu, ora),
                         "l1_rho_vs_exact": g_all, "l1_rho_vs_exact_near_vortex": g_near,
                         "oracle_l1_rho_vs_exact": o_all, "oracle_l1_rho_vs_exact_near_vortex": o_near,
                         "status": status, "oracle_seconds": osec}
    for n in (512, 2048):
        prob = W.shu_vortex_seeded(n, t_end=2.0, vel=W.STABLE_VELOCITY)
        s = af.Solver(n, n, prob.dx, prob.dy, prob.gamma, prob.bc)
        s.set_state(*W.discretise_torch(prob, "cuda"))
        absq = np.abs(W.discretise(prob)[0]).sum(axis=(1, 2)) * prob.dx * prob.dy if n <= 2048 else None
        tot = [s.totals()]
        t, k, failed = 0.0, 0, None
        while t < 2.0 * (1 - 1e-12) and k < 20000:
            speed = s.max_speed()
            if not speed > 0.0 or not np.isfinite(speed):
                failed = f"wave speed {speed} at step {k}, t = {t:.6g}"
                break
            dt = min(prob.cfl * prob.dx / speed, 2.0 - t)
            s.step(dt)
            t += dt
            k += 1
            if n == 2048:
                tot.append(s.totals())
        status = s.status()
        if failed:
            s.close()
            out[f"{n}^2"] = {"failed": failed, "status": status, "steps": k, "t": t}
            continue
        rho = s.get_state()[0][0].double().cpu().numpy()
        s.close()
        e_all, e_near = _vortex_l1_vs_exact(W, prob, rho, t)
        rec = {"t": t, "steps": k, "l1_rho_vs_exact": e_all, "l1_rho_vs_exact_near_vortex": e_near,
               "status": status}
        if n == 2048:
            tot = np.array(tot)
            rec["drift_per_step_max"] = float((np.abs(np.diff(tot, axis=0)) / absq).max())
            rec["drift_total"] = [float(x) for x in np.abs(tot[-1] - tot[0]) / absq]
        out[f"{n}^2"] = rec
    # the default background (1, 1) lies in the band where the scheme
    # amplifies perturbations: the same sweep at 512^2 blows up before t = 2
    prob = W.shu_vortex_seeded(512, t_end=2.0)
    s = af.Solver(512, 512, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*W.discretise_torch(prob, "cuda"))
    sp0, t, k, blow = s.max_speed(), 0.0, 0, None
    while t < 2.0 * (1 - 1e-12) and k < 4000:
        speed = s.max_speed()
        if not np.isfinite(speed) or speed > 3.0 * sp0:
            blow = {"step": k, "t": t, "max_speed": speed if np.isfinite(speed) else None}
            break
        dt = min(prob.cfl * prob.dx / speed, 2.0 - t)
        s.step(dt)
        t += dt
        k += 1
    s.close()
    out["background_1_1_512^2"] = {"blow_up": blow, "steps": k, "t": t,
                                    "note": "velocity (1, 1): Mach 1.2 along the diagonal, inside the band of "
                                            "oblique supersonic states that the scheme amplifies"}
    # and with (0.5, 0.5): the quadrant where the swirl adds to the motion
    # reaches the band
    prob = W.shu_vortex_seeded(1024, t_end=2.0, vel=(0.5, 0.5))
    s = af.Solver(1024, 1024, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*W.discretise_torch(prob, "cuda"))
    sp0, t, k, blow = s.max_speed(), 0.0, 0, None
    while t < 2.0 * (1 - 1e-12) and k < 6000:
        speed = s.max_speed()
        if not np.isfinite(speed) or speed > 3.0 * sp0:
            blow = {"step": k, "t": t, "max_speed": speed if np.isfinite(speed) else None}
            break
        dt = min(prob.cfl * prob.dx / speed, 2.0 - t)
        s.step(dt)
        t += dt
        k += 1
    s.close()
    out["background_0.5_0.5_1024^2"] = {"blow_up": blow, "steps": k, "t": t}
    n = 8192
    prob = W.shu_vortex_seeded(n, vel=W.STABLE_VELOCITY)
    s = af.Solver(n, n, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*W.discretise_torch(prob, "cuda"))
    t0 = s.totals()
    dt = prob.cfl * prob.dx / s.max_speed()
    s.run(seg_steps, dt)
    t1 = s.totals()
    status = s.status()
    rho = s.get_state()[0][0]
    s.close()
    mass = float(np.abs(t0[0]))
    e_all, e_near = _vortex_l1_vs_exact(W, prob, rho.double().cpu().numpy(), seg_steps * dt)
    out["8192^2"] = {"t": seg_steps * dt, "steps": seg_steps, "fixed_dt": dt, "l1_rho_vs_exact": e_all,
                     "l1_rho_vs_exact_near_vortex": e_near, "status": status,
                     "mass_drift_total": abs(float(t1[0] - t0[0])) / mass}
    out["note"] = ("standing vortex of the seed-2508 law (a moving one is unstable in long runs, see "
                   "background_1_1_512^2 and background_0.5_0.5_1024^2); "
                   "mean |rho - rho_exact| over cell averages, whole box and within 2.5 of the vortex centre; "
                   "the vortex is not periodic: its minimum-image data have a kink at distance 5 from the "
                   "centre (size about eps e^-12 / 2 pi, 3e-5 in velocity), whose waves set the whole-box "
                   "floor; FP32 point values set a second floor near 1e-7 at the finest grids")
    return out


def run_batch_leg(args, torch, af, W):
    """Seeded ensemble of 256 grids of 64^2 to 512^2 cells (half isentropic
    vortices, half four-quadrant Riemann problems) advanced by one graph
    launch of ``--batch-steps`` batched steps, tile height autotuned; cell
    updates counted per instance from the steps each one actually took."""
    probs = W.ensemble(256, seed=4096)
    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs], bcs=[p.bc for p in probs])
    for k, p in enumerate(probs):
        for key, v in p.options.items():
            b.set_option(key, v, k)
        b.set_state(k, *W.discretise_torch(p, "cuda"))
    cells = [p.nx * p.ny for p in probs]
    tile_h, tune_ms = b.autotune()
    b.run(args.warmup)
    _, steps0, _, _ = b.query()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.run(args.batch_steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    _, steps1, active, status = b.query()
    updates = int(sum(int(c) * (int(a) - int(z)) for c, a, z in zip(cells, steps1, steps0)))
    b.close()
    kinds = ["vortex" if k % 2 == 0 else "riemann" for k in range(len(probs))]
    stopped = [k for k in range(len(probs)) if status[k] & af.ST_STOPPED or not active[k]]
    return {
        "workload": "ensemble of 256 grids, N x N with N = round(64 * 8^U), U ~ U[0,1) from seed 4096; "
                    "even: isentropic vortex (centre, strength in [3,6]), odd: four-quadrant Riemann "
                    "(transmissive, Alg. 2, Alg. 3, Sec. 3.4 blend, flux limiter)",
        "instances": len(probs), "cells": int(sum(cells)), "steps": args.batch_steps,
        "value": updates / (ms / 1e3), "unit": UNIT, "ms": ms, "cell_updates": updates,
        "graph_launches": (args.batch_steps + 255) // 256, "tile_h": tile_h,
        "autotune_ms_per_launch": tune_ms,
        "stopped": {"vortex": sum(kinds[k] == "vortex" for k in stopped),
                    "riemann": sum(kinds[k] == "riemann" for k in stopped)},
        "note": "four-quadrant instances run with Alg. 2, Alg. 3, the Sec. 3.4 blend and the flux limiter; "
                "an instance whose state loses a finite wave speed stops",
    }


def _train_surrogate(args, af, W, probs, seed):
    """Both networks, trained on the GPU from (features, exact targets) pairs
    sampled from a batched ensemble of the given small problems."""
    import torch

    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs], bcs=[p.bc for p in probs])
    for k, p in enumerate(probs):
        for key, v in p.options.items():
            b.set_option(key, v, k)
        b.set_state(k, *W.discretise_torch(p, "cuda"))
    b.set_sampler(600000, 1200000, seed=seed, rate=0.08)
    b.run(12)
    Xv, Tv, _, Xe, Te, _ = (t.clone() for t in b.samples())
    b.close()
    nets = []
    for X, T in ((Xv, Tv), (Xe, Te)):
        m = af.Mlp(seed=5)
        m.fit_scales(X, T)
        hist = m.train(X, T, steps=args.surr_train_steps, batch=4096, lr=2e-3, seed=3)
        nets.append((m, float(hist[:10].mean()), float(hist[-10:].mean())))
    torch.cuda.synchronize()
    return nets, int(Xv.shape[0]), int(Xe.shape[0])


def _surrogate_full(args, torch, af, W, prob, nets, t_end, surr_opts=None):
    """Plain path and surrogate + exact fallback on the full-size grid from
    the same state to t_end: the plain run takes dt = cfl h / (its max speed)
    each step (the last one clipped); the surrogate run takes the same dt
    sequence, or its own CFL dt where that is smaller, until it reaches t_end.
    Each run is timed with CUDA events around all its steps (the per-step
    max-speed reads included, as in the plain run)."""
    dev = W.discretise_torch(prob, "cuda")
    plain = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options=prob.options)
    surr = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options=prob.options)
    surr.set_surrogate(nets[0], nets[1])
    for k, v in (surr_opts or {}).items():
        surr.set_option(k, v)
    h = min(prob.dx, prob.dy)
    for s in (plain, surr):  # warm-up steps, then the initial state again
        s.set_state(*dev)
        s.run(args.warmup, prob.cfl * h / s.max_speed())
        s.set_state(*dev)
        s.status()
    del dev
    surr.surrogate_stats(reset=True)
    stream = torch.cuda.current_stream()
    runs = {}
    dts = []
    for name, s in (("plain", plain), ("surrogate", surr)):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        t, k = 0.0, 0
        while t < t_end * (1 - 1e-12) and k < 20000:
            speed = s.max_speed()
            if not speed > 0.0 or speed == float("inf"):
                runs["failed"] = f"{name}: wave speed {speed} at step {k}, t = {t:.6g}"
                break
            dt = prob.cfl * h / speed
            if name == "surrogate" and k < len(dts):
                dt = min(dt, dts[k])
            dt = min(dt, t_end - t)
            s.step(dt)
            if name == "plain":
                dts.append(dt)
            t += dt
            k += 1
        ev1.record(stream)
        torch.cuda.synchronize()
        runs[name] = (ev0.elapsed_time(ev1), k, s.status())
        if "failed" in runs:
            break
    n_net, n_fall = surr.surrogate_stats()
    a, c = surr.get_state(), plain.get_state()
    rel = 0.0
    for x, y in zip(a, c):
        for v in (0, 3):  # density and energy / pressure: no vanishing components
            rel = max(rel, float((x[v].double() - y[v].double()).abs().sum() / y[v].double().abs().sum()))
    for s in (plain, surr):
        s.close()
    cells = prob.nx * prob.ny
    if "failed" in runs:
        return {"grid": [prob.nx, prob.ny], "final_time": t_end, "failed": runs["failed"],
                "status": sst_or_none(runs, "surrogate"), "plain_status": sst_or_none(runs, "plain")}
    (pm, pk, pst), (sm, sk, sst) = runs["plain"], runs["surrogate"]
    allowed = af.ST_FLUX_LIMITED
    out = {"grid": [prob.nx, prob.ny], "final_time": t_end, "steps_plain": pk, "steps_surrogate": sk,
           "value": cells * sk / (sm / 1e3), "plain_value": cells * pk / (pm / 1e3), "unit": UNIT,
           "ms_per_step": sm / sk, "plain_ms_per_step": pm / pk,
           "speedup_vs_plain": (cells * sk / sm) / (cells * pk / pm),
           "rel_l1_vs_plain": rel, "fallback_fraction": n_fall / max(1, n_net + n_fall),
           "status": sst, "plain_status": pst}
    bad = (pst | sst) & ~allowed
    if bad:
        out["failed"] = f"status bits {bad} other than AF_ST_FLUX_LIMITED"
    return out


def sst_or_none(runs, name):
    return runs[name][2] if name in runs else None


def _surrogate_vs_oracle(torch, af, W, ref, nets, vortex, surr_opts=None):
    """Plain and surrogate GPU runs at the oracle's size, with the oracle's dt
    sequence, against the FP64 oracle at its final time."""
    prob, ora, dts, osec = ref
    plain, pst, _ = _gpu_replay(torch, af, W, prob, dts)
    surr, sst, frac = _gpu_replay(torch, af, W, prob, dts, nets, surr_opts)
    rp, rs = _rel_l1(plain, ora), _rel_l1(surr, ora)
    out = {"grid": [prob.nx, prob.ny], "final_time": float(sum(dts)), "steps": len(dts),
           "rel_l1_plain_vs_oracle": rp, "rel_l1_surrogate_vs_oracle": rs,
           "surrogate_within_2x_of_plain": bool(rs <= 2.0 * rp), "surrogate_fallback_fraction": frac,
           "status": sst, "plain_status": pst, "oracle_seconds": osec,
           "norm": "relative L1, all arrays (averages and the three point-value arrays), worst variable"}
    if vortex:
        t = float(sum(dts))
        out["l1_rho_vs_exact"] = {"oracle": _vortex_l1_vs_exact(W, prob, ora[0][0], t)[0],
                                  "plain": _vortex_l1_vs_exact(W, prob, plain[0][0], t)[0],
                                  "surrogate": _vortex_l1_vs_exact(W, prob, surr[0][0], t)[0]}
    return out


# the Riemann case keeps the network away from shocks and contacts: its value
# is used only where every variable's range over the node's stencil is at
# most 0.05 in the features' scaled units (AF_OPT_SURR_SMOOTH)
RIEMANN_SURR = {"surr_smooth": 0.05}


def run_surrogate_leg(args, torch, af, W, refs):
    """Learned surrogate + exact fallback (K5): the 4096^2 isentropic vortex
    (seed 5) to t = --vortex-t and the 2048^2 four-quadrant problem (seed 6)
    to t = --riemann-t, each against the plain path on the same grid, and
    both paths against the FP64 oracle at an oracle-sized grid of the same
    law (256^2; the vortex of seed 2508 to t = 2, the four-quadrant problem of
    seed 6 to --riemann-t).  Networks are trained here, on the GPU, from
    samples of small seeded problems of each kind."""
    import numpy as np

    t0 = time.perf_counter()
    rng = np.random.default_rng(17)
    probs = [W.shu_vortex_seeded(int(rng.integers(64, 129)), seed=200 + k, t_end=np.inf, vel=W.STABLE_VELOCITY)
             for k in range(16)]
    nets, nv, ne = _train_surrogate(args, af, W, probs, seed=23)
    train_s = time.perf_counter() - t0
    n = args.surr_grid
    pair = (nets[0][0], nets[1][0])
    out = _surrogate_full(args, torch, af, W, W.shu_vortex_seeded(n, seed=5, vel=W.STABLE_VELOCITY), pair,
                          args.vortex_t)
    if refs:
        out["oracle_check"] = _surrogate_vs_oracle(torch, af, W, refs["vortex256"], pair, vortex=True)
    out.update({
        "workload": f"standing isentropic vortex, periodic [0,10]^2, {n}x{n} cells, centre and "
                    f"strength from seed 5, "
                    f"CFL 0.3, dt from the max speed every step, to t = {args.vortex_t}",
        "network": "64-128-128-128-16 GELU, BF16 weights, tcgen05 MMA with FP32 accumulation",
        "training": {"samples_vertex": nv, "samples_edge": ne,
                     "steps": args.surr_train_steps, "batch": 4096, "seconds_incl_sampling": train_s,
                     "loss_first_last_vertex": [nets[0][1], nets[0][2]],
                     "loss_first_last_edge": [nets[1][1], nets[1][2]],
                     "data": "16 seeded standing vortices of 64^2 to 128^2, 12 batched steps, "
                             "8% of nodes sampled"},
    })
    for m, _, _ in nets:
        m.close()
    # the Riemann case
    t0 = time.perf_counter()
    probs = [W.four_quadrant(int(rng.integers(64, 129)), seed=300 + k) for k in range(16)]
    nets, nv, ne = _train_surrogate(args, af, W, probs, seed=29)
    train_s = time.perf_counter() - t0
    nr = args.surr_grid // 2
    pair = (nets[0][0], nets[1][0])
    rie = _surrogate_full(args, torch, af, W, W.four_quadrant(nr, seed=6), pair, args.riemann_t, RIEMANN_SURR)
    if refs:
        rie["oracle_check"] = _surrogate_vs_oracle(torch, af, W, refs["riemann256"], pair, vortex=False,
                                                   surr_opts=RIEMANN_SURR)
    rie.update({
        "workload": f"four-quadrant Riemann problem, transmissive [0,1]^2, {nr}x{nr} cells, states from seed 6, "
                    f"Alg. 2, Alg. 3 with node bounds, Sec. 3.4 blend, flux limiter, Ubar = C2P of the average, "
                    f"CFL 0.3, dt from the max speed every step, to t = {args.riemann_t}",
        "surrogate_options": RIEMANN_SURR,
        "training": {"samples_vertex": nv, "samples_edge": ne, "seconds_incl_sampling": train_s,
                     "loss_first_last_vertex": [nets[0][1], nets[0][2]],
                     "loss_first_last_edge": [nets[1][1], nets[1][2]],
                     "data": "16 seeded four-quadrant problems of 64^2 to 128^2, 12 batched steps, 8% of nodes sampled"},
    })
    for m, _, _ in nets:
        m.close()
    out["riemann"] = rie
    return out


def run_reference(args):
    rank, world, _ = dist_setup()
    if rank != 0:
        return
    n = args.grid
    w = OracleWindow(n)
    for _ in range(args.warmup):
        w.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w.step()
    el = time.perf_counter() - t0
    value = w.cells * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n), "grid": [n, n], "cells": w.cells,
                   "sample": f"{w.window}x{w.window}-cell window of the {n}x{n} grid around the vortex "
                             f"(outflow ghosts at its edge): {w.cells} cells timed per step, not the full grid"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": w.threads, "kind": "oracle",
                         "sample": w.describe(n, args.steps) + ", one step per bench step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=8192, help="cells per side (default: 8192)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip every leg that runs the FP64 oracle on the host (CPU baseline, accuracy, "
                         "convergence, the surrogate leg's oracle checks)")
    ap.add_argument("--batch-steps", type=int, default=200,
                    help="steps of the batched-ensemble leg (0: skip it)")
    ap.add_argument("--no-surrogate", dest="surrogate", action="store_false",
                    help="skip the surrogate leg (K5: surrogate vs plain vs FP64 oracle at a final time)")
    ap.add_argument("--no-convergence", dest="convergence", action="store_false",
                    help="skip the convergence leg (K2: vortex sweep 128^2 to 8192^2)")
    ap.add_argument("--surr-steps", type=int, default=None, help="0: skip the surrogate leg (as --no-surrogate)")
    ap.add_argument("--surr-grid", type=int, default=4096, help="cells per side of the surrogate leg's vortex")
    ap.add_argument("--vortex-t", type=float, default=0.25, help="final time of the surrogate leg's vortex")
    ap.add_argument("--riemann-t", type=float, default=0.05, help="final time of the surrogate leg's Riemann case")
    ap.add_argument("--surr-train-steps", type=int, default=2000, help="Adam steps per surrogate network")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.surr_steps == 0:
        args.surrogate = False
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
