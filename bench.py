#!/usr/bin/env python3
"""Benchmark of the MacLAB step on GB300 (prints ONE JSON line on rank 0).

Workload (default): 3D lid-driven cavity, D3Q19, 128^3 nodes including the
wall shell, FP32 storage (drho = rho - 1, u / e), Re = 100 (lid speed
Re / (6 * 127) in lattice units), synthetic start from rest.  One benchmark
"step" is ``--inner`` MacLAB time steps (default 100) through the C ABI
(``maclab_step``).  The L2 cache is flushed (a 256 MiB write) before every
timed step, outside the timed interval; each step is timed with CUDA events on
the stream the kernels run on.

``value`` is MLUPS = fluid lattice-node updates per second / 1e6, summed over
ranks.  Extra keys: ``roofline`` of the dominant step kernel, ``cpu_baseline``
(the FP64 CPU oracle on a bounded sample), ``e2e`` (the same rate with host
buffers copied in and out every step), ``fp64`` (the same workload in FP64
storage), ``gpu_launches`` and ``clocks``.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, FP32 D3Q19 128³ vs FP64; adjoint/forward time"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--side", type=int, default=128, help="cavity side (nodes, walls included)")
    p.add_argument("--lattice", default="d3q19", choices=["d3q19", "d2q9"],
                   help="d2q9: the 2D lid-driven cavity of the same side instead (diagnostic runs)")
    p.add_argument("--case", default="cavity", choices=["cavity", "tgv"],
                   help="tgv: the periodic 3D Taylor-Green field (u0 = 0.02) of the same side instead "
                        "(diagnostic runs, D3Q19)")
    p.add_argument("--re", type=float, default=100.0)
    p.add_argument("--inner", type=int, default=100, help="MacLAB steps per benchmark step")
    p.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16", "f16"])
    p.add_argument("--no-extras", action="store_true", help="skip fp64 / e2e / cpu legs")
    p.add_argument("--kernel", default="auto", choices=["auto", "reference", "tiled", "folded", "segment", "rows2", "block"])
    p.add_argument("--ty", type=int, default=0, help="tiled kernel: rows per tile (0 = default)")
    p.add_argument("--tz", type=int, default=0, help="tiled kernel: planes per block (0 = default)")
    p.add_argument("--replicas", action="store_true",
                   help="N > 1: independent replicas instead of one domain split into slabs")
    p.add_argument("--halo", type=int, default=8, help="N > 1 slabs: ghost planes per side (exchange period)")
    p.add_argument("--leg", default="main", choices=["main", "adjoint", "batch", "lbm", "diag"],
                   help="adjoint / batch: run only that leg and print its JSON (for profiling)")
    return p.parse_args()


# ---------------------------------------------------------------- helpers

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" in r[5 + j]
                          and "Not" not in r[5 + j]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def traffic_from_profiles(kernel_tag, source_hash):
    """DRAM bytes per launch recorded by an ncu capture (profiles/*.md), if the
    kernel source has not changed since (same hash)."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, name)).read()
        m_tag = re.search(r"^kernel_tag:\s*(\S+)", txt, re.M)
        m_hash = re.search(r"^source_sha256:\s*(\S+)", txt, re.M)
        m_tr = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt, re.M)
        if m_tag and m_hash and m_tr and m_tag.group(1) == kernel_tag:
            return float(m_tr.group(1)) if m_hash.group(1) == source_hash else None
    return None


def step_source_hash():
    h = hashlib.sha256()
    for f in ("step.cu", "step_tiled.cuh", "step_tiled.cu", "step_fold.cuh", "step_fold.cu", "lattice.cuh",
              "common.cuh", "step_rows2.cuh", "step_rows2.cu"):
        with open(os.path.join(ROOT, "paper_1901_02716_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cavity_case(n, re):
    from paper_1901_02716_gb300 import inputs
    return inputs.cavity3d(n, lid=inputs.lid_speed(re, n))


# ---------------------------------------------------------------- CPU oracle leg

def oracle_rate(n, re, budget_s=10.0, max_steps=None, threads=0):
    """FP64 CPU oracle MLUPS on the same cavity, on `threads` host threads (0:
    every core this process may use); steps chosen to fill ~budget_s."""
    from oracle import oracle as orc
    used = orc.set_threads(threads if threads > 0 else orc.host_cores())
    case = cavity_case(n, re)
    rho, u = case.rho.copy(), case.u.copy()
    t0 = time.perf_counter()
    rho, u = orc.step(case.lattice, rho, u, case.periodic, wall=case.wall_mask)
    t1 = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(t1, 1e-6)))
    if max_steps:
        steps = min(steps, max_steps)
    t0 = time.perf_counter()
    rho, u = orc.step(case.lattice, rho, u, case.periodic, wall=case.wall_mask, nsteps=steps)
    dt = time.perf_counter() - t0
    return case.n_fluid * steps / dt / 1e6, steps, dt, used


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as orc
    cores = orc.set_threads(orc.host_cores())
    case = cavity_case(args.side, args.re)
    rho, u = case.rho.copy(), case.u.copy()
    for _ in range(args.warmup):
        rho, u = orc.step(case.lattice, rho, u, case.periodic, wall=case.wall_mask)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rho, u = orc.step(case.lattice, rho, u, case.periodic, wall=case.wall_mask)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = case.n_fluid * args.steps / total / 1e6
    sample = (f"{args.steps} MacLAB steps of the {args.side}^3 D3Q19 cavity (one per benchmark "
              f"step), FP64 CPU oracle on {cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"3D lid-driven cavity D3Q19 {args.side}^3, Re={args.re:g}",
                   "inner_steps": 1, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm, N > 1

def run_slabs(args, rank, world, local_rank):
    """One 128^3-per-rank cavity of 128 x 128 x (128 N) nodes split into N slabs
    along z (weak scaling): every rank steps its slab with the library and
    swaps `--halo` ghost planes with its neighbours over NCCL every `--halo`
    steps.  value = fluid updates of the whole domain / max-over-ranks time."""
    import torch
    import torch.distributed as dist
    from paper_1901_02716_gb300 import _build, inputs, slabs
    from paper_1901_02716_gb300 import maclab as M

    torch.cuda.set_device(local_rank)
    if not os.path.exists(M.library_path()):
        _build.build()
    prec = M.PRECISION_NAMES[args.precision]
    case = inputs.cavity3d(args.side, lid=inputs.lid_speed(args.re, args.side), nz=args.side * world)
    stream = torch.cuda.current_stream()
    sl = slabs.DistributedSlab(case, lambda sub: slabs.SolverStepper(sub, prec), depth=args.halo)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        sl.step(args.inner)
    torch.cuda.synchronize()
    dist_barrier(world)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    per = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sl.step(args.inner)
        b.record(stream)
        torch.cuda.synchronize()
        per.append(a.elapsed_time(b))
    dist_barrier(world)
    clocks = sampler.stop() if sampler else None
    total_ms = dist_max(sum(per), world)
    value = case.n_fluid * args.inner * args.steps / (total_ms * 1e-3) / 1e6
    # end to end: each rank's slab state in from and out to pinned host buffers every step
    sub = sl.sub
    rho_h = torch.from_numpy(sub.rho.astype(np.float32)).pin_memory()
    u_h = torch.from_numpy(sub.u.astype(np.float32)).pin_memory()
    s = sl.stepper.solver
    torch.cuda.synchronize()
    dist_barrier(world)
    t0 = time.perf_counter()
    k = max(2, min(args.steps, 5))
    for _ in range(k):
        s.set_state(rho_h.numpy(), u_h.numpy())
        sl.exchange()
        sl.step(args.inner)
        s.get_state_into(rho_h.numpy(), u_h.numpy())
    e2e_s = dist_max(time.perf_counter() - t0, world)
    nbytes = (rho_h.numel() + u_h.numel()) * 4
    kinfo = s.kernel_info()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"3D lid-driven cavity D3Q19 {args.side}x{args.side}x{args.side * world} "
                                   f"(walls included), Re={args.re:g}, {args.precision} storage",
                       "inner_steps": args.inner, "fluid_nodes": case.n_fluid,
                       "l2": "flushed (256 MiB write) before each timed step",
                       "parallelism": f"slabs x{world} along z, {args.halo} ghost planes per side, NCCL"},
            "gpu_launches": int(s.launches_per_step() * args.inner * args.steps),
            "kernel": kinfo["name"], "clocks": clocks,
            "e2e": {"value": case.n_fluid * args.inner * k / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": nbytes * world, "d2h_bytes_per_step": nbytes * world},
        }
        print(json.dumps(line), flush=True)
    s.close()


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1901_02716_gb300 import _build
    from paper_1901_02716_gb300 import maclab as M

    torch.cuda.set_device(local_rank)
    if not os.path.exists(M.library_path()):
        _build.build()
    prec = M.PRECISION_NAMES[args.precision]
    if args.lattice == "d2q9":
        from paper_1901_02716_gb300 import inputs
        case = inputs.cavity2d(args.side, lid=inputs.lid_speed(args.re, args.side))
    elif args.case == "tgv":
        from paper_1901_02716_gb300 import inputs
        case = inputs.tgv3d(args.side, 0.02)
    else:
        case = cavity_case(args.side, args.re)
    stream = torch.cuda.current_stream()
    solver = M.Solver.from_case(case, prec, stream=ctypes_stream(stream))
    solver.set_kernel({"auto": M.KERNEL_AUTO, "reference": M.KERNEL_REFERENCE,
                       "tiled": M.KERNEL_TILED, "folded": M.KERNEL_FOLDED,
                       "segment": M.KERNEL_SEGMENT, "rows2": M.KERNEL_ROWS2,
                       "block": M.KERNEL_BLOCK}[args.kernel])
    if args.ty or args.tz:
        solver.set_tile(args.ty, args.tz)
    lups_per_step = case.n_fluid * args.inner
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step():
        solver.step(args.inner)

    # warm-up
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    dist_barrier(world)

    sampler = ClockSampler(local_rank) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))                 # evict the state from L2 (not timed)
        ev[i][0].record(stream)
        one_step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks = sampler.stop() if sampler else None
    per = [a.elapsed_time(b) for a, b in ev]          # ms
    total_ms = sum(per)
    total_ms = dist_max(total_ms, world)
    value = world * lups_per_step * args.steps / (total_ms * 1e-3) / 1e6
    launches_per_step = solver.launches_per_step() * args.inner
    avg_launch_ms = total_ms / (args.steps * launches_per_step)

    if rank != 0:
        solver.close()
        return

    d = case.d
    bytes_per_lup = (d + 1) * 2 * {"f32": 4, "f64": 8, "bf16": 2, "f16": 2}[args.precision]
    steps_per_launch = solver.steps_per_launch()
    algo_bytes = bytes_per_lup * case.n_fluid * steps_per_launch
    peak, peak_kind = peaks()
    achieved = algo_bytes / (avg_launch_ms * 1e-3) / 1e9
    kernel_tag = solver.kernel_tag()
    traffic = traffic_from_profiles(kernel_tag, step_source_hash())

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": (f"periodic 3D Taylor-Green field D3Q19 {args.side}^3, u0=0.02, "
                                f"{args.precision} storage" if d == 3 and args.case == "tgv" else
                                (f"3D lid-driven cavity D3Q19 {args.side}^3" if d == 3 else
                                 f"2D lid-driven cavity D2Q9 {args.side}^2") +
                                f" (walls included), Re={args.re:g}, {args.precision} storage"),
                   "inner_steps": args.inner, "fluid_nodes": case.n_fluid,
                   "l2": "flushed (256 MiB write) before each timed step",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "dram_gbs_measured": (traffic / (avg_launch_ms * 1e-3) / 1e9) if traffic else None,
                     "kernel": kernel_tag, "bytes_per_lup": bytes_per_lup,
                     "peak_kind": peak_kind, "avg_launch_us": avg_launch_ms * 1e3},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clocks,
    }

    if not args.no_extras and d == 3:  # the 2D cavity line is a diagnostic run without the extra legs
        # the arithmetic ceiling beside the memory roofline: algorithmic flops
        # per update (D3Q19 ~200, D2Q9 ~80) against the measured paired-FP32 rate
        fpl = 200 if d == 3 else 80
        fp_peak = M.maclab_measure_fp32_peak()
        fp_ach = value * 1e6 * fpl / 1e12
        line["fp32"] = {"flops_per_lup": fpl, "achieved_tflops": fp_ach, "peak_tflops": fp_peak,
                        "frac": fp_ach / fp_peak if fp_peak > 0 else None,
                        "peak_kind": "measured (paired FP32 FMA chains, maclab_measure_fp32_peak)"}
        line["suite"] = suite_leg(M, stream)
        line["e2e"] = e2e_leg(M, case, prec, args, stream)
        line["adjoint_forward"] = adjoint_leg(M, case, prec, args, stream)
        # the differentiable workload: periodic 96^3 Taylor-Green field with the seeded perturbation
        from paper_1901_02716_gb300 import inputs
        line["adjoint_forward_tgv96"] = adjoint_leg(M, inputs.tgv3d(96, 0.02, 1e-3, 5), prec, args, stream)
        line["diagnostics"] = diagnostics_leg(M, case, prec, stream)
        if args.precision != "f64":
            line["fp64"] = fp64_leg(M, case, args, stream, flush)
        mlups, steps, secs, cores = oracle_rate(args.side, args.re)
        mlups1, steps1, secs1, _ = oracle_rate(args.side, args.re, budget_s=8.0, threads=1)
        line["cpu_baseline"] = {
            "value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} MacLAB steps of the same {args.side}^3 cavity from rest "
                      f"({secs:.1f} s, FP64, {cores} host threads)",
            "one_core": {"value": mlups1, "unit": "MLUPS", "cores": 1,
                         "sample": f"{steps1} steps ({secs1:.1f} s, FP64, one thread)"}}
    solver.close()
    print(json.dumps(line), flush=True)


def ctypes_stream(stream):
    return stream.cuda_stream if stream.cuda_stream else None


def e2e_leg(M, case, prec, args, stream):
    """Same MLUPS through the public API with host buffers: pinned host (rho, u)
    in, ``inner`` steps, (rho, u) back to pinned host, every step."""
    import torch
    grid = case.grid
    rho_h = torch.empty(grid, dtype=torch.float32).pin_memory()
    u_h = torch.empty((3,) + grid, dtype=torch.float32).pin_memory()
    rho_h.copy_(torch.from_numpy(case.rho.astype(np.float32)))
    u_h.copy_(torch.from_numpy(case.u.astype(np.float32)))
    rho_n, u_n = rho_h.numpy(), u_h.numpy()
    s = M.Solver.from_case(case, prec, stream=ctypes_stream(stream))
    k = max(2, min(args.steps, 5))
    for _ in range(2):
        s.set_state(rho_n, u_n)
        s.step(args.inner)
        s.get_state_into(rho_n, u_n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        s.set_state(rho_n, u_n)
        s.step(args.inner)
        s.get_state_into(rho_n, u_n)           # synchronises
    dt = time.perf_counter() - t0
    s.close()
    nbytes = rho_h.numel() * 4 + u_h.numel() * 4
    return {"value": case.n_fluid * args.inner * k / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}


def adjoint_leg(M, case, prec, args, stream):
    """Time of one reverse step of a rollout (maclab_adjoint_step_nu: the
    reverse step with its viscosity term; states already stored) against one
    forward step, same workload and storage type; beside it the reverse step
    without the term and the per-node viscosity kernel alone."""
    import torch
    s = M.Solver.from_case(case, prec, stream=ctypes_stream(stream))
    nb = s.state_bytes()
    s0 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s1 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s.step(20)
    s.get_lattice_state(s0)
    s.step(1)
    s.get_lattice_state(s1)
    ab = s.adjoint_bytes()
    lam = [torch.zeros(ab, dtype=torch.uint8, device="cuda") for _ in range(2)]
    gf = torch.zeros(3, dtype=torch.float64, device="cuda")
    k = 20

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(k):
            fn(i)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    nu_acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    t_fwd = timed(lambda i=0: s.step(1))
    t_adj = timed(lambda i=0: M.maclab_adjoint_step(s.handle, s0, s1, lam[i & 1], lam[(i + 1) & 1], gf))
    t_nu = timed(lambda i=0: M.maclab_adjoint_nu_term(s.handle, s0, lam[i & 1], nu_acc, s1))

    def pair(i=0):  # a reverse step of a rollout that differentiates nu: the term, then the step
        M.maclab_adjoint_nu_term(s.handle, s0, lam[i & 1], nu_acc, s1)
        M.maclab_adjoint_step(s.handle, s0, s1, lam[i & 1], lam[(i + 1) & 1], gf)

    t_pair = timed(pair)
    s.close()
    return {"forward_ms": t_fwd, "adjoint_ms": t_adj, "ratio": t_adj / t_fwd,
            "adjoint_launches_per_step": 1, "nu_term_ms": t_nu,
            "adjoint_with_nu_ms": t_pair, "ratio_with_nu_gradient": t_pair / t_fwd,
            "ratio_with_nu_gradient_separate": (t_adj + t_nu) / t_fwd}


def diagnostics_leg(M, case, prec, stream):
    """The FP64 diagnostics reduction (mass, kinetic energy, momentum, residual:
    both state buffers read once) on the same workload, three ways: its added
    device time inside a running step loop (k steps each followed by
    maclab_diagnostics_device, minus k steps alone: the cost of monitoring every
    step), its device time alone (back to back, state resident in L2), and the
    wall time of the synchronous maclab_diagnostics call (the reduction plus
    the round trip to the host).  The memory roofline is taken on the in-loop
    figure."""
    import torch
    s = M.Solver.from_case(case, prec, stream=ctypes_stream(stream))
    s.step(3)
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    for _ in range(3):
        s.diagnostics()
        M.maclab_diagnostics_device(s.handle, out)
    torch.cuda.synchronize()
    k = 64

    def monitored(n):
        for _ in range(n):
            s.step(1)
            M.maclab_diagnostics_device(s.handle, out)

    def diag_only(n):
        for _ in range(n):
            M.maclab_diagnostics_device(s.handle, out)

    step_ms = _timed_steps(torch, stream, s.step, k) / k
    both_ms = _timed_steps(torch, stream, monitored, k) / k
    alone_ms = _timed_steps(torch, stream, diag_only, k) / k
    t0 = time.perf_counter()
    for _ in range(k):
        s.diagnostics()
    call_ms = (time.perf_counter() - t0) * 1e3 / k
    nbytes = 2 * s.state_bytes()
    s.close()
    in_loop = max(both_ms - step_ms, 1e-6)
    gbs = nbytes / (in_loop * 1e-3) / 1e9
    return {"ms": in_loop, "ms_alone": alone_ms, "call_ms": call_ms, "step_ms": step_ms,
            "bytes": nbytes, "gbs": gbs, "frac": gbs / peaks()[0]}


def _timed_steps(torch, stream, step, n, reps=3):
    """Device time (ms) of `n` steps, best of `reps`, after one warm-up call."""
    step(n)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(n)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best = t if best is None else min(best, t)
    return best


def suite_leg(M, stream):
    """The other configurations of the workload set, FP32, state L2/HBM resident
    as it naturally is (no flush inside the timed steps): MLUPS each.  Grids
    whose steps take microseconds are timed over whole 32-step graphs."""
    import torch
    from paper_1901_02716_gb300 import inputs
    out = {}
    # batched 2D cavities: 64 sides in {64..512}, Re log-uniform [100, 3200]
    sides, res, lids = inputs.batch_cavity_sides(64, seed=4)
    cases = [inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)]
    b = M.Batch.from_cases(cases, M.F32, stream=ctypes_stream(stream))
    rows = b.tune()
    info = b.info()
    n = 256
    ms = _timed_steps(torch, stream, b.step, n)
    out["batch_64_cavities"] = {"mlups": info["fluid_nodes"] * n / (ms * 1e-3) / 1e6,
                                "fluid_nodes": info["fluid_nodes"], "rows_per_item": rows,
                                "launches_per_step": info["launches_per_step"],
                                "steps_per_launch": info["steps_per_launch"],
                                "work_items": info["items"]}
    # the same work list in one persistent launch per call (depth 3), whatever the tuner chose
    try:
        b.set_depth(3)
    except M.MacLABError as err:  # the cooperative launch does not fit this device
        out["batch_64_cavities_persistent"] = {"unavailable": str(err)}
    else:
        info = b.info()
        ms = _timed_steps(torch, stream, b.step, n)
        b.sync()
        out["batch_64_cavities_persistent"] = {"mlups": info["fluid_nodes"] * n / (ms * 1e-3) / 1e6,
                                               "rows_per_item": info["rows"],
                                               "launches_per_call": 1 + n - 2 * ((n - 1) // 2),
                                               "work_items": info["items"]}
    b.close()
    # the stream-and-collide comparator (SRT-BGK D2Q9, tau = 0.8) beside MacLAB on
    # the same periodic 1024^2 Taylor-Green field: traffic and state per update
    tg = inputs.tgv2d(1024, 0.02)
    lb = M.Lbm(1024, 1024, 0.8, M.F32, stream=ctypes_stream(stream))
    lb.set_state(tg.rho, tg.u)
    n = 640
    ms = _timed_steps(torch, stream, lb.step, n)
    li = lb.info()
    lb.close()
    s = M.Solver.from_case(tg, M.F32, stream=ctypes_stream(stream))
    s.tune()
    ms_m = _timed_steps(torch, stream, s.step, n)
    mi = s.kernel_tag()
    s.close()
    lb_mlups = li["nodes"] * n / (ms * 1e-3) / 1e6
    mac_mlups = tg.n_fluid * n / (ms_m * 1e-3) / 1e6
    out["srt_lbm_vs_maclab_2d_1024"] = {
        "lbm_mlups": lb_mlups, "lbm_bytes_per_update": li["bytes_per_update"],
        "lbm_state_bytes": li["state_bytes"],
        "lbm_hbm_frac_algorithmic": lb_mlups * 1e6 * li["bytes_per_update"] / (peaks()[0] * 1e9),
        "maclab_mlups": mac_mlups, "maclab_bytes_per_update": 24, "maclab_kernel": mi,
        "maclab_state_bytes": 2 * 3 * 4 * tg.n_fluid, "speedup": mac_mlups / lb_mlups}
    for name, case, steps, prec in (
            ("cavity2d_1024", inputs.cavity2d(1024, lid=inputs.lid_speed(1000.0, 1024)), 640, M.F32),
            ("cavity2d_256", inputs.cavity2d(256, lid=inputs.lid_speed(100.0, 256)), 1280, M.F32),
            ("cavity3d_128_bf16", cavity_case(128, 100.0), 100, M.BF16_STORE),
            ("tgv3d_96", inputs.tgv3d(96, 0.02), 128, M.F32),
            ("cavity2d_8192_hbm", inputs.cavity2d(8192, lid=inputs.lid_speed(1000.0, 8192)), 20, M.F32),
            ("cavity3d_512_hbm", inputs.cavity3d(512, lid=inputs.lid_speed(100.0, 512)), 10, M.F32),
            ("cavity3d_512_bf16_hbm", inputs.cavity3d(512, lid=inputs.lid_speed(100.0, 512)), 10, M.BF16_STORE)):
        s = M.Solver.from_case(case, prec, stream=ctypes_stream(stream))
        tile = s.tune()
        ms = _timed_steps(torch, stream, s.step, steps)
        bpl = (4 if prec == M.BF16_STORE else 8) * (case.d + 1)
        mlups = case.n_fluid * steps / (ms * 1e-3) / 1e6
        out[name] = {"mlups": mlups, "fluid_nodes": case.n_fluid, "kernel": s.kernel_tag(),
                     "tile_ty_tz": list(tile) if tile is not None else None,
                     "hbm_frac_algorithmic": mlups * 1e6 * bpl / (peaks()[0] * 1e9)}
        s.close()
        del case
    # obstacle workload: 128 x 128 x 256 channel with a sphere spinning about the
    # axis (per-node wall velocity), walls from an explicit byte mask: 32 B of
    # state + 1 B of mask per update
    case, field = inputs.channel3d_sphere(spin=0.01)
    s = M.Solver.from_case(case, M.F32, stream=ctypes_stream(stream))
    s.set_wall_state(np.ones(case.grid), field)
    tile = s.tune()
    ms = _timed_steps(torch, stream, s.step, 50)
    mlups = case.n_fluid * 50 / (ms * 1e-3) / 1e6
    out["channel3d_sphere_128x128x256"] = {
        "mlups": mlups, "fluid_nodes": case.n_fluid, "kernel": s.kernel_tag(),
        "tile_ty_tz": list(tile) if tile is not None else None, "bytes_per_lup": 33,
        "hbm_frac_algorithmic": mlups * 1e6 * 33 / (peaks()[0] * 1e9)}
    s.close()
    return out


def fp64_leg(M, case, args, stream, flush):
    import torch
    s = M.Solver.from_case(case, M.F64, stream=ctypes_stream(stream))
    for _ in range(2):
        s.step(args.inner)
    ts = []
    for i in range(3):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(args.inner)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    s.close()
    return {"value": case.n_fluid * args.inner * 3 / (sum(ts) * 1e-3) / 1e6, "unit": "MLUPS",
            "bytes_per_lup": 64}


# ---------------------------------------------------------------- distributed plumbing

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("MACLAB_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_leg(args):
    """One leg alone, on one GPU: the reverse step or the FP64 diagnostics on the
    configured cavity, the 64 batched cavities, or the SRT-BGK comparator on
    the periodic 1024^2 Taylor-Green field; prints the leg's JSON."""
    import torch
    from paper_1901_02716_gb300 import _build
    from paper_1901_02716_gb300 import maclab as M
    torch.cuda.set_device(0)
    if not os.path.exists(M.library_path()):
        _build.build()
    stream = torch.cuda.current_stream()
    if args.leg == "adjoint":
        from paper_1901_02716_gb300 import inputs
        case = inputs.tgv3d(args.side, 0.02, 1e-3, 5) if args.case == "tgv" else cavity_case(args.side, args.re)
        out = adjoint_leg(M, case, M.PRECISION_NAMES[args.precision], args, stream)
    elif args.leg == "diag":
        out = diagnostics_leg(M, cavity_case(args.side, args.re), M.PRECISION_NAMES[args.precision], stream)
    elif args.leg == "lbm":
        from paper_1901_02716_gb300 import inputs
        tg = inputs.tgv2d(1024, 0.02)
        lb = M.Lbm(1024, 1024, 0.8, M.F32, stream=ctypes_stream(stream))
        lb.set_state(tg.rho, tg.u)
        ms = _timed_steps(torch, stream, lb.step, 640)
        li = lb.info()
        lb.close()
        mlups = li["nodes"] * 640 / (ms * 1e-3) / 1e6
        out = {"mlups": mlups, "bytes_per_update": li["bytes_per_update"],
               "hbm_frac_algorithmic": mlups * 1e6 * li["bytes_per_update"] / (peaks()[0] * 1e9)}
    else:
        from paper_1901_02716_gb300 import inputs
        sides, res, lids = inputs.batch_cavity_sides(64, seed=4)
        b = M.Batch.from_cases([inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)], M.F32,
                               stream=ctypes_stream(stream))
        rows = b.tune()
        info = b.info()
        ms = _timed_steps(torch, stream, b.step, 200)
        out = {"mlups": info["fluid_nodes"] * 200 / (ms * 1e-3) / 1e6, "rows_per_item": rows,
               "steps_per_launch": info["steps_per_launch"], "work_items": info["items"]}
        b.close()
    print(json.dumps({"leg": args.leg, **out}))


def main():
    args = parse()
    if args.leg != "main":
        run_leg(args)
        return
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif world > 1 and not args.replicas:
        run_slabs(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
