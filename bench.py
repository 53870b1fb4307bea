"""Throughput of the space-time multigrid slab solver on one GB300.

Workload (default): 3D heat equation on [0,1]^3, Q2 elements on 32^3 cells whose
interior vertices are jittered by U[-0.15h, 0.15h] (seed 11), dG(2) in time,
tau = 1/32 (32 slabs), diffusion piecewise constant on a 4x4x4 grid of blocks,
log-uniform in [1e-2, 1e2] (seed 12), source of u = sin(pi x) sin(pi y) sin(pi z) sin(pi t).
One step = one time slab: right-hand side, previous-slab initial guess, FGMRES
(FP64) preconditioned by one FP32 V-cycle per iteration, to ||r|| <= 1e-8 ||b||.
Metric: space-time DoFs (unconstrained, N_t x interior nodes) solved per second.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "space-time DoFs/s solved to 1e-8 rel. residual (mixed FP32 V-cycle in FP64 FGMRES)"
UNIT = "DoF/s"


def workload(n_cells=32, p=2, k=2, n_slabs=32):
    return dict(name=f"heat3d_q{p}_dg{k}_{n_cells}cubed_jitter0.15_rho4blocks", dim=3, N=n_cells, p=p, k=k,
                tau=1.0 / n_slabs, n_slabs=n_slabs, vertices=synth.jittered_vertices(n_cells, 3),
                rho=synth.block_coefficient(n_cells, 3, blocks=4))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ----------------------------------------------------------------------------- oracle timing
def oracle_sample(n_cells: int, n_slabs: int, tau: float):
    """Oracle slab marching (assembly, sparse LU once, one solve per slab) on an n_cells^3 sample."""
    from oracle import slab, space
    t0 = time.perf_counter()
    V = synth.jittered_vertices(n_cells, 3)
    rho = synth.block_coefficient(n_cells, 3, blocks=2)
    g = space.Grid(n_cells, 3, 2, V)
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, rho), "heat", "dg", 2, tau)
    X = g.node_coords()
    u_prev = np.zeros(g.n_nodes)
    for n in range(n_slabs):
        f = np.stack([synth.heat_sine_source(X, tau * (n + th)) for th in prob.sys.tw.nodes])
        u = prob.solve(prob.rhs(f, None, u_prev))
        u_prev = u[-1]
    dt = time.perf_counter() - t0
    dofs = prob.nt * int((~prob.bmask).sum())
    return dofs * n_slabs / dt, dofs, dt


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_cells, tau = 10, 1.0 / 32
    from oracle import slab, space
    V = synth.jittered_vertices(n_cells, 3)
    rho = synth.block_coefficient(n_cells, 3, blocks=2)
    g = space.Grid(n_cells, 3, 2, V)
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, rho), "heat", "dg", 2, tau)
    X = g.node_coords()
    dofs = prob.nt * int((~prob.bmask).sum())
    u_prev = np.zeros(g.n_nodes)

    def step(n):
        nonlocal u_prev
        f = np.stack([synth.heat_sine_source(X, tau * (n + th)) for th in prob.sys.tw.nodes])
        u = prob.solve(prob.rhs(f, None, u_prev))
        u_prev = u[-1]

    for n in range(args.warmup):
        step(n)
    t0 = time.perf_counter()
    for n in range(args.steps):
        step(args.warmup + n)
    dt = time.perf_counter() - t0
    value = dofs * args.steps / dt
    sample = (f"oracle slab marching (sparse LU factorised in the warm-up, one triangular solve per slab) on "
              f"the same workload family at 10^3 cells (Q2, dG(2), jitter 0.15h, 2^3 coefficient blocks), "
              f"{dofs} DoFs per slab")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "heat3d_q2_dg2_10cubed_jitter0.15_rho2blocks (oracle sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_kernel_only(args):
    """Profiling helper: builds the workload's hierarchy with fixed relaxation weights (no Arnoldi)
    and launches one kernel a few times; used for ncu captures of a single kernel."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    wl = workload(args.n_cells)
    ctx = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                       vcycle_precision=stmg.FP32, omega=[0.2] * 16)
    kind, prec = {"apply64": (stmg.KERNEL_APPLY, stmg.FP64), "apply32": (stmg.KERNEL_APPLY, stmg.FP32),
                  "asm32": (stmg.KERNEL_ASM, stmg.FP32), "asm64": (stmg.KERNEL_ASM, stmg.FP64),
                  "vcycle32": (stmg.KERNEL_VCYCLE, stmg.FP32)}[args.only_kernel]
    ms = ctx.time_kernel(kind, 0, prec, reps=args.steps)
    print(json.dumps({"kernel": args.only_kernel, "avg_launch_ms": ms, "workload": wl["name"]}))
    ctx.close()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2408_04372_gb300 as stmg
    stmg.load()

    wl = workload(args.n_cells)
    vprec = stmg.FP64 if args.plain else stmg.FP32
    ctx = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                       vcycle_precision=vprec, rtol=1e-8, restart=30, max_it=200)
    nt, nn = ctx.nt, ctx.n_nodes
    X = ctx.node_coords()
    from paper_2408_04372_gb300 import DG  # noqa: F401
    tn = radau_nodes(wl["k"])
    n_slabs = wl["n_slabs"]
    interior = (wl["N"] * wl["p"] - 1) ** 3
    dofs_per_step = nt * interior
    # all sources resident on the device before timing
    F = torch.empty((n_slabs, nt * nn), dtype=torch.float64, device=dev)
    for s in range(n_slabs):
        f = np.stack([synth.heat_sine_source(X, wl["tau"] * (s + th)) for th in tn])
        F[s].copy_(torch.from_numpy(f.reshape(-1)))
    rhs = torch.empty(nt * nn, dtype=torch.float64, device=dev)
    u = torch.empty_like(rhs)
    u_prev = torch.zeros(nn, dtype=torch.float64, device=dev)
    its = []

    def step(i):
        s = i % n_slabs
        if s == 0:
            u_prev.zero_()
        ctx.rhs(F[s], rhs, u0=u_prev)
        ctx.guess_previous(u_prev, u)
        st = ctx.solve(rhs, u)
        if not st["converged"]:
            raise RuntimeError(f"slab {s} did not converge: {st}")
        its.append(st["iterations"])
        u_prev.copy_(u[(nt - 1) * nn:])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    its.clear()
    launches0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record()
        for i in range(args.steps):
            step(args.warmup + i)
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    ms, value = aggregate_replicas(ms, dofs_per_step, args.steps, world, dev)

    # end to end through the C ABI from pinned host buffers (H2D of f and u0, D2H of u each step)
    Fh = torch.empty((n_slabs, nt * nn), dtype=torch.float64).pin_memory()
    Fh.copy_(F.cpu())
    uh = torch.zeros(nt * nn, dtype=torch.float64).pin_memory()
    u0h = torch.zeros(nn, dtype=torch.float64).pin_memory()
    Fn, un, u0n = Fh.numpy(), uh.numpy().reshape(nt, nn), u0h.numpy()
    e2e_steps = max(1, min(args.steps, 8))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        s = (args.warmup + i) % n_slabs
        if s == 0:
            u0n[:] = 0.0
        ctx.solve_slab_host(Fn[s].reshape(nt, nn), u0n, out_u=un)
        u0n[:] = un[nt - 1]
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * dofs_per_step * e2e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": int(8 * (nt * nn + nn)), "d2h_bytes_per_step": int(8 * nt * nn)}

    # dominant kernel: the FP64 operator apply on the finest level (one per FGMRES iteration)
    roof = None
    cpu = None
    extra = {}
    if rank == 0:
        apply_ms = ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.FP64, reps=20)
        asm_ms = ctx.time_kernel(stmg.KERNEL_ASM, 0, stmg.FP32, reps=20)
        vc_ms = ctx.time_kernel(stmg.KERNEL_VCYCLE, 0, vprec, reps=10)
        n = wl["p"] + 1
        cells = wl["N"] ** 3
        flops_unit = 12 * n ** 4 + (16 + 8 * nt) * n ** 3          # per cell and time DoF
        flops = flops_unit * cells * nt
        peaks = read_peaks()
        fp64_peak = 1.25e12
        roof = {"kernel": "apply3d_kernel<N=3,NT=3,double> (finest level, FP64)", "bound": "alu",
                "achieved": flops / (apply_ms * 1e-3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": flops / (apply_ms * 1e-3) / fp64_peak, "traffic": read_traffic("apply_fp64"),
                "peak_source": "FP64 1.25 TFLOP/s nominal (GB300 table; no measured FP64 peak)",
                "avg_launch_ms": apply_ms}
        asm_bytes = cells * nt * (n ** 3) ** 2 * 4 + 2 * 4 * nt * nn
        extra["asm_fp32_finest"] = {"avg_launch_ms": asm_ms, "algorithmic_bytes": asm_bytes,
                                    "achieved_GBs": asm_bytes / (asm_ms * 1e-3) / 1e9,
                                    "frac_of_measured_hbm": asm_bytes / (asm_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        extra["vcycle_ms"] = vc_ms
        if not args.skip_cpu:
            v, d, dt = oracle_sample(10, 4, wl["tau"])
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"oracle marching of 4 slabs (assembly + sparse LU + 4 solves, {dt:.1f} s) of the same "
                             f"workload family at 10^3 cells ({d} DoFs per slab)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32" if not args.plain else "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "cells": wl["N"] ** 3, "p": wl["p"], "time": f"dG({wl['k']})",
                       "dofs_per_step": dofs_per_step, "rtol": 1e-8, "vcycle": "fp64" if args.plain else "fp32",
                       "parallelism": f"replicas{world}", "l2": "working set > L2 (inverses alone 0.29 GB)",
                       "fgmres_iterations_mean": float(np.mean(its)) if its else None},
            "gpu_launches": int(launches), "clocks": clk.summary(), "e2e": e2e, "roofline": roof,
            "cpu_baseline": cpu, "kernels": extra}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def aggregate_replicas(ms_local, dofs_per_step, steps, world, device):
    """Replicas only: slowest rank's time, every rank's DoFs.  Returns (max ms, whole-job DoF/s)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * dofs_per_step * steps / (ms / 1e3)


def radau_nodes(k):
    """Right Gauss-Radau nodes on [0,1] (time nodes of dG(k)); roots of P_k - P_{k+1}."""
    from numpy.polynomial import legendre as L
    if k == 0:
        return np.array([1.0])
    c = np.zeros(k + 2)
    c[k], c[k + 1] = 1.0, -1.0
    x = np.sort(np.real(L.legroots(c)))
    x[-1] = 1.0
    return 0.5 * (x + 1.0)


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def read_traffic(key):
    """DRAM bytes per launch from the committed ncu capture; None once the kernel source changed."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(key)
    if d is None:
        return None
    src = os.path.join(ROOT, d["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != d["source_sha"]:
        return None
    return d.get("bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-cells", type=int, default=32)
    ap.add_argument("--plain", action="store_true", help="FP64 V-cycle (plain STMG) instead of mixed precision")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--only-kernel", default=None, choices=["apply64", "apply32", "asm32", "asm64", "vcycle32"],
                    help="profiling helper: time one kernel only (fixed omega, no Arnoldi)")
    args = ap.parse_args()
    if args.only_kernel:
        return run_kernel_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
