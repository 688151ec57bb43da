#!/usr/bin/env python
"""Throughput benchmark: lattice updates per second of the fused stream-collide
step on GB300, mixed-precision batched form (headline) against the plain FP64
form, with the roofline of the dominant kernel and the FP64 CPU oracle timed on
the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Workload (headline): 256 periodic Taylor-Green domains of uneven size (sides
uniform in 32..512, seed 20260101), MJ fifth-order equilibrium, tau swept
0.55..2.0, amplitudes 0.005..0.05 c, FP32 populations stored as deviations
from each domain's rest equilibrium, one launch per step over
a tile work list, autotuned grid, steps replayed from a CUDA graph. Under
torchrun the batch's domains are split over the ranks by cell count (strong
scaling; --scaling weak gives every rank its own seeded batch instead). Ranks
share no data: only the timing (max) and the cell count (sum) are reduced, and
rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1709_09073_gb300 import partition, workloads as W  # noqa: E402

METRIC = "lattice updates/s (MLUPS) FP64 vs mixed+batched on 1 GB300; % roofline"
UNIT = "MLUPS"
BYTES_PER_CELL = {0: 1152, 1: 576, 2: 288, 3: 288, 4: 576}   # 2 x 72 x element size
STORAGE_NAME = {0: "f64", 1: "f32", 2: "bf16dev", 3: "f16dev", 4: "f32dev"}
# the mixed step's variants (rlbm_select_kernel) by the kernel each launches
KERNEL_NAMES = {0: "k_step_mixed", 1: "k_step_mixed_tma"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and ids[min(local, len(ids) - 1)].strip().isdigit():
        return int(ids[min(local, len(ids) - 1)])
    return local


def timed_steps(sim, steps, torch):
    """Device time (s) of `steps` steps with CUDA events on the handle's stream."""
    s = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    sim.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def rank_workload(rank, world=1, scaling="strong"):
    """The batch one rank advances. strong: the one 256-domain batch split over
    the ranks by cell count (longest first, to the least-loaded rank), so the
    total work is fixed as the rank count grows; weak: every rank its own
    independently seeded batch, so the per-rank work is fixed. The domains are
    independent problems either way: ranks share no data."""
    if scaling == "weak":
        return W.batched_taylor_green(seed=20260101 + rank)
    return partition.shard(W.batched_taylor_green(seed=20260101), rank, world)


def over_ranks(x, world, torch, op="max", device="cuda"):
    """Max (timings) or sum (cells) of a scalar over all ranks; metadata only."""
    if world == 1:
        return x
    import torch.distributed as dist
    v = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(v.item())


def barrier_max(t, world, torch):
    return over_ranks(t, world, torch, "max")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def traffic_record(kernel):
    """DRAM bytes per cell of `kernel` from the committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        return d.get(kernel)
    except ValueError:
        return None


def run_native(args):
    import torch
    from paper_1709_09073_gb300 import build, rlbm
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    rlbm.load()
    pipes = rlbm.pipe_peaks()  # measured FMA-chain throughput: the ALU ceilings of the roofline
    wl = rank_workload(rank, world, args.scaling)
    cells = wl.cells
    total_cells = over_ranks(cells, world, torch, "sum")  # units all ranks process per step
    storage = rlbm.RLBM_F32DEV
    sim, st0 = rlbm.from_workload(wl, storage=storage)
    grid = sim.tune(3)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index(local))
    barrier(world)
    sampler.start()
    t = timed_steps(sim, args.steps, torch)
    clocks = sampler.stop()
    barrier(world)
    t = barrier_max(t, world, torch)
    status = sim.sync_status()
    value = total_cells * args.steps / t / 1e6
    per_launch = t / args.steps
    bpc = BYTES_PER_CELL[storage]
    achieved = bpc * cells / per_launch / 1e9
    hbm_peak, peak_kind = peaks()
    kname = KERNEL_NAMES[sim.select_kernel()]
    tr = traffic_record("%s_f32dev_mj" % kname)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4),
                "traffic": round(tr * cells) if tr else None,
                "peak_source": peak_kind, "kernel": "%s<MJ, F32Dev>" % kname,
                "algorithmic_bytes_per_cell": bpc}
    launches = sim.last_step_info()[1]

    # end to end through the public API with host buffers: the packed fields of
    # every domain copied from pinned host memory and initialised in one call
    # (rlbm_init_all), every step followed by a status read-back, the packed
    # fields n, theta, u of every domain read back (rlbm_moments_all) into
    # pinned memory;
    # the device buffers they pass through are allocated before the clock starts
    pinned = [torch.from_numpy(np.concatenate([getattr(s, k).reshape(-1) for s in wl.init])).pin_memory()
              for k in ("a", "theta", "ux", "uy")]
    dev_in = [torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(4)]
    dev_out = [torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(4)]  # n, theta, ux, uy
    out_host = [torch.empty(cells, dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_steps = max(1, args.steps)  # the K steps of the device-timed region
    kind = wl.init[0].kind

    def e2e_once():
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, h in zip(dev_in, pinned):
            d.copy_(h, non_blocking=True)
        sim.init_all(kind, *dev_in)
        for _ in range(e2e_steps):
            sim.step(1)
            sim.sync_status()
        sim.moments_all(out=dev_out)
        for o, h in zip(dev_out, out_host):
            h.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        return barrier_max(time.perf_counter() - t0, world, torch)

    # three repetitions, each from a fresh initialisation; the median is reported
    reps = sorted(e2e_once() for _ in range(3))
    te = reps[1]
    h2d = 4 * 8 * cells
    d2h = 4 * 8 * cells + 4 * e2e_steps
    e2e = {"value": round(total_cells * e2e_steps / te / 1e6, 2), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps),
           "steps": e2e_steps,
           "reps_value": [round(total_cells * e2e_steps / r / 1e6, 2) for r in reps],
           "what": "median of 3: packed fields from pinned host -> rlbm_init_all -> "
                   "(rlbm_step(1) + status read) x K -> rlbm_moments_all (n, theta, u) -> pinned host"}
    sim.close()
    del sim, dev_in, dev_out

    # the plain FP64 form on the same workload (the comparison the metric names)
    fp64 = None
    if not args.no_fp64:
        sim64, _ = rlbm.from_workload(wl, storage=rlbm.RLBM_F64)
        sim64.tune(1)
        sim64.step(max(1, args.warmup // 10))
        k64 = max(2, args.steps // 20)
        barrier(world)
        t64 = barrier_max(timed_steps(sim64, k64, torch), world, torch)
        v64 = total_cells * k64 / t64 / 1e6
        flops_per_cell = FP64_FLOPS_PER_CELL
        alu_peak = pipes["fp64_flops"] / 1e12
        instr_peak = pipes["fp64_flops"] / 2 / 1e9  # DFMA, DADD and DMUL issue at one rate
        ach = flops_per_cell * cells / (t64 / k64) / 1e12
        ach_i = FP64_INSTR_PER_CELL * cells / (t64 / k64) / 1e9
        fp64 = {"value": round(v64, 2), "unit": UNIT, "steps": k64,
                "ms_per_step": round(t64 / k64 * 1e3, 3),
                "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": round(alu_peak, 4),
                             "unit": "TFLOP/s (FP64)", "frac": round(ach / alu_peak, 4),
                             "flops_per_cell": flops_per_cell,
                             "peak_source": "measured: FP64 FMA-chain kernel on all %d SMs (rlbm_pipe_peaks)"
                                            % pipes["sm_count"]},
                # the pipe issues DADD and DMUL at the DFMA rate but they carry one
                # flop: the instruction throughput of the FP64 pipe is its real bound
                "fp64_pipe": {"instr_per_cell": FP64_INSTR_PER_CELL, "achieved": round(ach_i, 1),
                              "peak": round(instr_peak, 1), "unit": "G instr/s",
                              "frac": round(ach_i / instr_peak, 4)},
                "hbm_achieved_gbs": round(1152 * cells / (t64 / k64) / 1e9, 1)}
        sim64.close()

    others = None
    if world == 1 and not args.no_extra:
        others = run_other_configs(args, hbm_peak)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(wl, budget_s=args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t / args.steps * 1e3, 4), "higher_is_better": True,
                "scaling": args.scaling, "vs_baseline": None,
                "dtype": "f32 (double-float totals, Landau residual, n, eps; no FP64 instruction)",
                "data": "synthetic",
                "config": {"workload": wl.name, "domains": len(wl.domains), "cells_per_gpu": cells,
                           "cells_all_ranks": int(total_cells),
                           "sides": ("uniform 32..512 (seed 20260101), split over ranks by cell count"
                                     if args.scaling == "strong" else "uniform 32..512 (seed 20260101 + rank)"),
                           "tau": "0.55..2.0",
                           "u0": "0.005..0.05", "edf": "MJ", "order": 5,
                           "storage": "f32dev (FP32 populations as relative deviations from the rest equilibrium)",
                           "grid": grid, "l2": "inputs larger than L2 (%.1f GB of populations)"
                           % (2 * 288 * cells / 1e9),
                           "parallelism": ("one batch, whole domains per GPU by cell count (no collective)"
                                           if args.scaling == "strong" else
                                           "an independent batch per GPU (no collective)")},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64": fp64, "other_configs": others, "status": status,
                "pipe_peaks": {"fp64_tflops": round(pipes["fp64_flops"] / 1e12, 4),
                               "fp32_tflops": round(pipes["fp32_flops"] / 1e12, 3),
                               "sm_count": pipes["sm_count"], "how": "rlbm_pipe_peaks: FMA chains, best of 3"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# FP64 operations per cell update of the plain kernel (k_step_f64<MJ>), FMA = 2:
# 872 DFMA + 308 DADD + 202 DMUL per cell, the executed-instruction counts ncu
# reports for one 1024^2 launch divided by its cells; used for the FP64 ALU
# roofline of the plain form.
FP64_FLOPS_PER_CELL = 2 * 872 + 308 + 202
FP64_INSTR_PER_CELL = 872 + 308 + 202


def _oracle_rate(O, wl, budget_s):
    """Cells per second of one oracle step over whole domains of the workload,
    in order, until the time budget is used; (rate, domains, cells)."""
    done_cells, t_used, ndom = 0, 0.0, 0
    for d, s in zip(wl.domains, wl.init):
        dom = O.domain(d.nx, d.ny, d.tau, d.edf, d.bc, d.t_wall)
        f, macro, _ = O.init(dom, s.kind, s.a, s.theta, s.ux, s.uy)
        t0 = time.perf_counter()
        O.step(dom, f, macro)
        t_used += time.perf_counter() - t0
        done_cells += d.nx * d.ny
        ndom += 1
        if t_used > budget_s:
            break
    return done_cells / t_used, ndom, done_cells


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_baseline(wl, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores (OpenMP over rows),
    and once more on one thread with a third of the budget."""
    from oracle import oracle as O
    O.build()
    cores = O.num_threads()
    rate, ndom, cells = _oracle_rate(O, wl, budget_s)
    O.set_num_threads(1)
    try:
        rate1, ndom1, cells1 = _oracle_rate(O, wl, budget_s / 3)
    finally:
        O.set_num_threads(cores)
    return {"value": round(rate / 1e6, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 step of each of the first %d domains (%d cells) of the workload" % (ndom, cells),
            "single_thread": {"value": round(rate1 / 1e6, 4), "unit": UNIT, "cores": 1,
                              "sample": "1 step of each of the first %d domains (%d cells)" % (ndom1, cells1)},
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


def run_profile_case(args):
    """A small case for ncu: init and a few steps of one kernel.
    mixed: 2048 x 2048 Taylor-Green, MJ, FP32 deviations (2.4 GB of populations);
    batch: the first 48 domains of the headline batch (4.5 M cells, 2.6 GB);
    fourier: the first 16 domains of the FD Fourier batch in BF16 deviations (4.2 M cells, 1.2 GB);
    fp64:  1024 x 1024 Taylor-Green, MJ, FP64 (1.2 GB). Inputs exceed L2."""
    import torch
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    if args.profile_case == "batch":  # the first 48 domains of the headline batch (4.5 M cells)
        storage = rlbm.RLBM_F32DEV
        full = W.batched_taylor_green()
        wl = W.Workload(full.name + "_first48", full.domains[:48], full.init[:48], 3)
    elif args.profile_case == "fourier":
        storage = rlbm.RLBM_BF16DEV
        full = W.batched_fourier()
        wl = W.Workload(full.name + "_first16", full.domains[:16], full.init[:16], 3)
    else:
        L, storage = (2048, rlbm.RLBM_F32DEV) if args.profile_case == "mixed" else (1024, rlbm.RLBM_F64)
        wl = W.taylor_green(L=L, u0=0.02, tau=0.9, steps=3)
    sim, _ = rlbm.from_workload(wl, storage=storage)
    if args.profile_case in ("mixed", "batch", "fourier"):
        sim.select_kernel({"l1": rlbm.RLBM_KERNEL_L1, "tma": rlbm.RLBM_KERNEL_TMA}[args.kernel])
    sim.step(3)
    torch.cuda.synchronize()
    t = timed_steps(sim, args.steps, torch) if args.steps > 0 else 0.0
    print(json.dumps({"profile_case": args.profile_case, "kernel": args.kernel, "cells": wl.cells,
                      "status": sim.sync_status(),
                      "steps": args.steps, "mlups": round(wl.cells * args.steps / t / 1e6, 1) if t else None}))


def run_other_configs(args, hbm_peak):
    """The other throughput configurations of the method on this GPU, each with
    its own autotuned launch: the 8192^2 Bose-Einstein hot spot in FP32
    deviations and in FP64, the 64-domain Fermi-Dirac Fourier-flow batch in the
    16-bit deviation storages (and in FP32 deviations, for comparison), and the
    headline batch in BF16 deviations. Device time with CUDA events over K steps
    after W warm-up steps; inputs exceed L2."""
    import torch
    from paper_1709_09073_gb300 import rlbm
    out = {}
    cases = [("hot_spot_8192x8192_BE_f32dev", W.hot_spot(L=8192), rlbm.RLBM_F32DEV, 20),
             ("hot_spot_8192x8192_BE_f64", None, rlbm.RLBM_F64, 4),
             ("fourier_x64_1024x256_FD_bf16dev", W.batched_fourier(), rlbm.RLBM_BF16DEV, 50),
             ("fourier_x64_1024x256_FD_f16dev", None, rlbm.RLBM_F16DEV, 50),
             ("fourier_x64_1024x256_FD_f32dev", None, rlbm.RLBM_F32DEV, 50),
             ("batched_taylor_green_x256_MJ_bf16dev", W.batched_taylor_green(), rlbm.RLBM_BF16DEV, 50)]
    wl = None
    for name, w, storage, k in cases:
        wl = w if w is not None else wl
        sim, st = rlbm.from_workload(wl, storage=storage)
        sim.tune(1)
        sim.step(3)
        t = timed_steps(sim, k, torch)
        st |= sim.sync_status()
        bpc = BYTES_PER_CELL[storage]
        ach = bpc * wl.cells / (t / k) / 1e9
        out[name] = {"value": round(wl.cells * k / t / 1e6, 2), "unit": UNIT, "steps": k,
                     "ms_per_step": round(t / k * 1e3, 3), "cells": wl.cells, "status": st,
                     "kernel": "k_step_f64" if storage == rlbm.RLBM_F64 else KERNEL_NAMES[sim.select_kernel()],
                     "hbm": {"achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                             "frac": round(ach / hbm_peak, 4), "algorithmic_bytes_per_cell": bpc}}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    whole = out["hot_spot_8192x8192_BE_f32dev"]
    out["hot_spot_8192x8192_BE_f32dev_2yslabs"] = run_slab_case(W.hot_spot(L=8192), rlbm.RLBM_F32DEV, 20, 2,
                                                                 whole["value"])
    return out


def run_slab_case(wl, storage, k, nslabs, whole_value):
    """The one-domain workload cut into `nslabs` y-slabs, held as domains of one
    handle on this GPU. Every step packs the edge rows of each slab, copies
    each face into its neighbour's receive buffer (the device copy standing in
    for the message between GPUs), unpacks them into the ghost rows and steps
    once. Reports the throughput, the exchange's own device time per step and
    the ratio to the undivided domain."""
    import dataclasses
    import torch
    from paper_1709_09073_gb300 import rlbm, slabs
    spec, init = wl.domains[0], wl.init[0]
    bounds = slabs.slab_bounds(spec.ny, nslabs)
    specs = [dataclasses.replace(spec, ny=y1 - y0, bc=slabs.slab_bcs(spec.bc, r, nslabs))
             for r, (y0, y1) in enumerate(bounds)]
    sim = rlbm.Simulation(specs, edf=spec.edf, storage=storage)
    st = 0
    for r, (y0, y1) in enumerate(bounds):
        cut = lambda a: np.ascontiguousarray(a[y0:y1])
        st |= sim.init(r, W.InitialState(init.kind, cut(init.a), cut(init.theta), cut(init.ux), cut(init.uy)))
    nb = [slabs.neighbours(r, nslabs, spec.bc[2] == W.PERIODIC) for r in range(nslabs)]
    send = [(sim.edge_row_buffer(r), sim.edge_row_buffer(r)) for r in range(nslabs)]
    recv = [(sim.edge_row_buffer(r), sim.edge_row_buffer(r)) for r in range(nslabs)]
    pick = lambda bufs, r: tuple(b if n is not None else None for b, n in zip(bufs, nb[r]))

    def exchange():
        for r in range(nslabs):
            sim.pack_edge_rows(r, *pick(send[r], r))
        for r, (below, above) in enumerate(nb):
            if below is not None:
                recv[r][0].copy_(send[below][1])
            if above is not None:
                recv[r][1].copy_(send[above][0])
            sim.unpack_ghost_rows(r, *pick(recv[r], r))

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        for _ in range(n):
            fn()
        e1.record(sim.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def step():
        exchange()
        sim.step(1)

    sim.tune(1)
    for _ in range(3):
        step()
    t = timed(step, k)
    t_ex = timed(exchange, k)  # idempotent: rewrites the ghost rows with the same rows
    st |= sim.sync_status()
    face_bytes = send[0][0].numel() * send[0][0].element_size()
    sim.close()
    del sim, send, recv
    torch.cuda.empty_cache()
    value = wl.cells * k / t / 1e6
    return {"value": round(value, 2), "unit": UNIT, "steps": k, "ms_per_step": round(t / k * 1e3, 3),
            "cells": wl.cells, "slabs": nslabs, "status": st,
            "exchange_us_per_step": round(t_ex / k * 1e6, 1),
            "face_bytes": face_bytes,
            "vs_undivided": round(value / whole_value, 4),
            "what": "per step: pack both edge rows of every slab, device copy to the neighbour, "
                    "unpack into the ghost rows, one step launch (no graph)"}


def run_reference(args):
    """The oracle as the reference arm: same metric, bounded sample per step."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    wl = W.batched_taylor_green(seed=20260101)
    # one bounded sample: the first domains up to ~0.6 M cells, one step each per "step"
    sample, cells = [], 0
    for d, s in zip(wl.domains, wl.init):
        sample.append((d, s))
        cells += d.nx * d.ny
        if cells > 600_000:
            break
    states = []
    for d, s in sample:
        dom = O.domain(d.nx, d.ny, d.tau, d.edf, d.bc, d.t_wall)
        f, macro, _ = O.init(dom, s.kind, s.a, s.theta, s.ux, s.uy)
        states.append([dom, f, macro])

    def one_step():
        for stt in states:
            f, mo, _ = O.step(stt[0], stt[1], stt[2])
            stt[1], stt[2] = f, mo[[0, 2, 3]].copy()

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    t = time.perf_counter() - t0
    value = cells * args.steps / t / 1e6
    sample_txt = "first %d domains of %s (%d cells), full step each" % (len(sample), wl.name, cells)
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "sample": sample_txt},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--scaling", choices=["strong", "weak"], default="strong",
                    help="strong: split the one batch over the ranks by cell count; "
                         "weak: an independently seeded batch per rank")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the hot-spot and Fourier-flow configurations")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--kernel", choices=["l1", "tma"], default="l1",
                    help="mixed step variant of --profile-case mixed")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured FP64/FP32 FMA throughput of the GPU and exit")
    ap.add_argument("--profile-case", choices=["mixed", "batch", "fourier", "fp64"], default=None,
                    help="run a small single-domain case for ncu instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.peaks:
        from paper_1709_09073_gb300 import build, rlbm
        build.build()
        rlbm.load()
        p = rlbm.pipe_peaks()
        print(json.dumps({"fp64_tflops": round(p["fp64_flops"] / 1e12, 4),
                          "fp32_tflops": round(p["fp32_flops"] / 1e12, 3), "sm_count": p["sm_count"]}))
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
