"""Throughput of the space-time multigrid slab solver on one GB300.

Workload (default): 3D heat equation on [0,1]^3, Q2 elements on 32^3 cells whose
interior vertices are jittered by U[-0.15h, 0.15h] (seed 11), dG(2) in time,
tau = 1/32 (32 slabs), diffusion piecewise constant on a 4x4x4 grid of blocks,
log-uniform in [1e-2, 1e2] (seed 12), source of u = sin(pi x) sin(pi y) sin(pi z) sin(pi t).
One step = one time slab: right-hand side, previous-slab initial guess, FGMRES (FP64)
preconditioned by one FP32 V-cycle per iteration, to ||r|| <= 1e-8 ||b||.  The line also reports
the plain FP64 solver on the same slabs ("compare").

--workload c5: the learned-initial-guess workload (Q2 on 48^3 Cartesian cells, dG(1), 256 slabs,
8 moving Gaussian sources): slabs 0-127 solved by the mixed solver train the 3D conv network,
slabs 128-255 are solved twice, from the learned guess (kept only when its FP64 residual is below
the previous-slab guess's) and from the previous-slab guess; iterations and wall time of both.
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
    """Samples nvidia-smi clocks and throttle reasons every 50 ms while running."""

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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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
ORACLE_SAMPLE_CELLS = 16   # oracle sample of the headline family: 16^3 cells (1/8 of the 32^3 grid)


def oracle_c2_run(n_cells, slabs, warmup):
    """The oracle's slab solve on the headline workload family at n_cells^3: the same jitter, the same
    4^3 coefficient blocks, Q2, dG(2), tau = 1/32; per slab the right-hand side, the previous-slab guess
    and FGMRES (rtol 1e-8) preconditioned by the oracle's V-cycle with the GPU arm's options (Schwarz sum
    weighted by the node multiplicity, omega = 1 on every level, hierarchy ending at the first level with
    at most 1500 unknowns).  Hierarchy set-up (assembly, local inverses) is timed apart.  Returns a dict."""
    from oracle import mg
    tau = 1.0 / 32
    t0 = time.perf_counter()
    V = synth.jittered_vertices(n_cells, 3)
    rho = synth.block_coefficient(n_cells, 3, blocks=4)
    H = mg.Hierarchy(3, n_cells, 2, 2, "heat", "dg", tau, V, rho_cell=rho, weighted=True, coarse_max_dofs=1500,
                     omegas=[1.0] * 16)
    setup_s = time.perf_counter() - t0
    prob = H.levels[0].prob
    X = prob.grid.node_coords()
    nn = prob.grid.n_nodes
    u_prev = np.zeros(nn)
    its = []

    def step(n):
        nonlocal u_prev
        f = np.stack([synth.heat_sine_source(X, tau * (n + th)) for th in prob.sys.tw.nodes])
        rhs = prob.rhs(f, None, u_prev).reshape(-1)
        res = mg.fgmres(lambda v: prob.S @ v, H.vcycle, rhs, np.tile(u_prev, prob.nt), rtol=1e-8)
        its.append(res.iterations)
        u_prev = res.x.reshape(prob.nt, nn)[-1].copy()

    for n in range(warmup):
        step(n)
    t1 = time.perf_counter()
    for n in range(slabs):
        step(warmup + n)
    dt = time.perf_counter() - t1
    dofs = prob.nt * int((~prob.bmask).sum())
    return {"value": dofs * slabs / dt, "unit": UNIT, "dofs_per_slab": dofs, "slabs": slabs, "solve_s": dt,
            "setup_s": setup_s, "fgmres_iterations_mean": float(np.mean(its[warmup:])),
            "threads": os.environ.get("OMP_NUM_THREADS", str(os.cpu_count()))}


def oracle_subprocess(n_cells, slabs, warmup, threads):
    """oracle_c2_run in a fresh interpreter with `threads` BLAS/OpenMP threads (spawned, not forked,
    so it is safe after CUDA initialisation in the parent)."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[var] = str(threads)
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-run", str(n_cells),
                          "--steps", str(slabs), "--warmup", str(warmup)],
                         env=env, capture_output=True, text=True, timeout=3600)
    if res.returncode != 0:
        raise RuntimeError(f"oracle run failed: {res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_sample_text(r, n_cells):
    return (f"oracle slab solves (FGMRES + the oracle's V-cycle, rtol 1e-8, {r['fgmres_iterations_mean']:.1f} "
            f"iterations) on the headline family at {n_cells}^3 cells ({r['dofs_per_slab']} DoFs per slab): "
            f"{r['slabs']} slabs in {r['solve_s']:.1f} s after warm-up, hierarchy set-up {r['setup_s']:.1f} s "
            f"excluded; scipy sparse products run on one thread whatever the BLAS thread count")


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_cells = ORACLE_SAMPLE_CELLS
    r = oracle_c2_run(n_cells, args.steps, args.warmup)
    one = oracle_subprocess(n_cells, 2, 1, 1)
    cores = os.cpu_count()
    wl_name = workload(n_cells)["name"]
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["solve_s"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl_name, "sample_of": workload(args.n_cells)["name"], "cells": n_cells ** 3,
                       "p": 2, "time": "dG(2)", "rtol": 1e-8, "dofs_per_step": r["dofs_per_slab"]},
            "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
                             "value_1_thread": one["value"], "sample": oracle_sample_text(r, n_cells)},
            "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_oracle_full(args):
    """The oracle on the full headline grid (32^3 cells), all host threads and one thread."""
    out = {}
    for threads in (os.cpu_count(), 1):
        out[f"threads_{threads}"] = oracle_subprocess(args.n_cells, 2, 1, threads)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "impl": "oracle", "config": {"workload": workload(args.n_cells)["name"]},
                      "runs": out}), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_net_only(args):
    """Profiling helper for the learned guess's tensor-core kernels: the learned-guess workload's grid
    (Q2 on 48^3 cells, dG(1): 97^3 nodes), the 4-60-60-60-2 network with seeded weights, `steps`
    inferences and training steps on seeded inputs; prints the mean times."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    N = args.n_cells if args.n_cells != 32 else 48
    ctx = stmg.Context(3, N, 2, 1, 1.0 / 256, omega=[0.2] * 8, vcycle_precision=stmg.FP32)
    nt, nn = ctx.nt, ctx.n_nodes
    channels = (2 * nt, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, nt)
    W, b = synth.conv_net_init(channels, seed=15)
    net = stmg.Net(ctx, channels, W, b, (1.0, 1.0, 1.0))
    up = torch.from_numpy(synth.random_vector(nt * nn, seed=31)).cuda()
    f = torch.from_numpy(synth.random_vector(nt * nn, seed=32)).cuda()
    g = torch.empty_like(up)
    times = {}
    for name, fn in (("predict", lambda: net.predict(up, f, g)), ("train_step", lambda: net.train_step(up, f, up, 1e-4))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name + "_ms"] = e0.elapsed_time(e1) / args.steps
    voxels = (N * 2 + 1) ** 3
    flops = 2 * 27 * voxels * sum(channels[l] * channels[l + 1] for l in range(len(channels) - 1))
    times["inference_tflops"] = flops / (times["predict_ms"] * 1e-3) / 1e12
    print(json.dumps({"workload": f"heat3d_q2_dg1_{N}cubed learned guess network", "channels": list(channels), **times}))
    net.close()
    ctx.close()
    return 0


def run_kernel_only(args):
    """Profiling helper: builds the workload's hierarchy with fixed relaxation weights (no Arnoldi)
    and launches one kernel a few times; used for ncu captures of a single kernel."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    if args.only_kernel == "net":
        return run_net_only(args)
    wl = workload(args.n_cells)
    ctx = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                       vcycle_precision=stmg.FP32, omega=[0.2] * 16, smoother_kind=smoother_kind(stmg, args),
                       inverse_precision={"fp32": stmg.FP32, "bf16": stmg.BF16, "fp64": stmg.FP64,
                                          "fp8": stmg.FP8}[args.inverse])
    kind, prec = {"apply64": (stmg.KERNEL_APPLY, stmg.FP64), "apply32": (stmg.KERNEL_APPLY, stmg.FP32),
                  "applydf": (stmg.KERNEL_APPLY, stmg.DF32),
                  "asm32": (stmg.KERNEL_ASM, stmg.FP32), "asm64": (stmg.KERNEL_ASM, stmg.FP64),
                  "vcycle32": (stmg.KERNEL_VCYCLE, stmg.FP32), "vcycle64": (stmg.KERNEL_VCYCLE, stmg.FP64),
                  "ortho64": (stmg.KERNEL_ORTHO, stmg.FP64), "orthodf": (stmg.KERNEL_ORTHO, stmg.DF32)}[args.only_kernel]
    ms = ctx.time_kernel(kind, args.level, prec, reps=args.steps)
    print(json.dumps({"kernel": args.only_kernel, "level": args.level, "avg_launch_ms": ms, "workload": wl["name"]}))
    ctx.close()
    return 0


NET_CHANNELS_HIDDEN = 60
TRAIN_SLABS = 16
TRAIN_EPOCHS = 40


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
    inv_prec = {"fp32": stmg.FP32, "bf16": stmg.BF16, "fp64": stmg.FP64, "fp8": stmg.FP8}[args.inverse] \
        if not args.plain else stmg.FP64
    ctx = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                       vcycle_precision=vprec, inverse_precision=inv_prec, rtol=1e-8, restart=30, max_it=200,
                       coarse_max_dofs=args.coarse_max_dofs, asm_weighting=args.asm_weighting,
                       outer_relax=args.outer_relax if not args.plain else 0, smoother_kind=smoother_kind(stmg, args))
    nt, nn = ctx.nt, ctx.n_nodes
    n = nt * nn
    X = ctx.node_coords()
    tn = radau_nodes(wl["k"])
    n_slabs = wl["n_slabs"]
    interior = (wl["N"] * wl["p"] - 1) ** 3
    dofs_per_step = nt * interior
    # sources of every slab resident in HBM before timing
    F = torch.empty((n_slabs, n), dtype=torch.float64, device=dev)
    for s in range(n_slabs):
        f = np.stack([synth.heat_sine_source(X, wl["tau"] * (s + th)) for th in tn])
        F[s].copy_(torch.from_numpy(f.reshape(-1)))
    sols = torch.zeros((n_slabs + 1, n), dtype=torch.float64, device=dev)   # sols[s + 1] = slab s; sols[0] = initial
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    cand = torch.empty(n, dtype=torch.float64, device=dev)
    use_net = args.net and not args.plain

    def solve_slab(s, u, net=None):
        prev = sols[s]
        prev_end = prev[(nt - 1) * nn:]
        ctx.rhs(F[s], rhs, u0=prev_end)
        ctx.guess_previous(prev_end, u)
        taken = False
        if net is not None:
            net.predict(prev, F[s], cand)
            taken = ctx.select_guess(rhs, cand, u)
        st = ctx.solve(rhs, u)
        if not st["converged"]:
            raise RuntimeError(f"slab {s} did not converge: {st}")
        sols[s + 1].copy_(u)
        return st, taken

    # learned guess: plain marching over the training slabs, then Adam on (previous slab, source) -> slab
    net, train_info = None, None
    u = torch.empty(n, dtype=torch.float64, device=dev)
    if use_net:
        t0 = time.perf_counter()
        for s in range(TRAIN_SLABS):
            solve_slab(s, u)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        su = 1.0 / float(sols[1:TRAIN_SLABS + 1].pow(2).mean().sqrt())
        sf = 1.0 / float(F[:TRAIN_SLABS].pow(2).mean().sqrt())
        incr = torch.stack([sols[s + 1] - sols[s][(nt - 1) * nn:].repeat(nt) for s in range(1, TRAIN_SLABS)])
        so = 1.0 / float(incr.pow(2).mean().sqrt())
        channels = (2 * nt, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, nt)
        W, b = synth.conv_net_init(channels, seed=15)
        net = stmg.Net(ctx, channels, W, b, (su, sf, so))
        t1 = time.perf_counter()
        losses = []
        for epoch in range(TRAIN_EPOCHS):
            for s in range(1, TRAIN_SLABS):
                losses.append(net.train_step(sols[s], F[s], sols[s + 1], 2e-3))
        torch.cuda.synchronize()
        train_info = {"slabs": TRAIN_SLABS - 1, "epochs": TRAIN_EPOCHS, "train_s": time.perf_counter() - t1,
                      "data_solve_s": t_solve, "loss_first_epoch": float(np.mean(losses[:TRAIN_SLABS - 1])),
                      "loss_last_epoch": float(np.mean(losses[-(TRAIN_SLABS - 1):])),
                      "params": int(sum(w.size for w in W) + sum(x.size for x in b)), "channels": list(channels)}
    first = TRAIN_SLABS if use_net else 0
    span = n_slabs - first

    def slab_of(i):
        return first + i % span

    its, taken, relaxed = [], [], []
    for i in range(args.warmup):
        solve_slab(slab_of(i), u, net)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record()
        for i in range(args.steps):
            st, tk = solve_slab(slab_of(args.warmup + i), u, net)
            its.append(st["iterations"])
            relaxed.append(st["relaxed_iterations"])
            taken.append(tk)
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    ms, value = aggregate_replicas(ms, dofs_per_step, args.steps, world, dev)

    # comparison arms on the same slabs (not the headline): mixed without the network, plain FP64
    compare = {}
    if rank == 0 and not args.skip_compare and not args.plain:
        def timed(fn, steps):
            torch.cuda.synchronize()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = [fn(slab_of(args.warmup + i)) for i in range(steps)]
            b_.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b_), out
        if use_net:
            k2 = min(args.steps, 8)
            t_m, o_m = timed(lambda s: solve_slab(s, u)[0], k2)
            compare["mixed_previous_slab_guess"] = {"value": dofs_per_step * k2 / (t_m / 1e3), "unit": UNIT,
                                                    "fgmres_iterations_mean": float(np.mean([x["iterations"] for x in o_m]))}
        ctx64 = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                             vcycle_precision=stmg.FP64, rtol=1e-8, restart=30, max_it=200,
                             coarse_max_dofs=args.coarse_max_dofs, asm_weighting=args.asm_weighting)
        def plain(s):
            prev_end = sols[s][(nt - 1) * nn:]
            ctx64.rhs(F[s], rhs, u0=prev_end)
            ctx64.guess_previous(prev_end, u)
            return ctx64.solve(rhs, u)
        plain(slab_of(args.warmup))
        k3 = min(args.steps, 4)
        t_p, o_p = timed(plain, k3)
        compare["plain_fp64_previous_slab_guess"] = {"value": dofs_per_step * k3 / (t_p / 1e3), "unit": UNIT,
                                                     "fgmres_iterations_mean": float(np.mean([x["iterations"] for x in o_p]))}
        ctx64.close()
        if not use_net:
            # the same solve with the other Schwarz sum (printed eq. vanka0 <-> weighted by node multiplicity)
            other = 1 - args.asm_weighting
            ctxw = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                                vcycle_precision=vprec, inverse_precision=inv_prec, rtol=1e-8, restart=30,
                                max_it=200, coarse_max_dofs=args.coarse_max_dofs, asm_weighting=other)
            ctxr = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                                vcycle_precision=vprec, inverse_precision=inv_prec, rtol=1e-8, restart=30,
                                max_it=200, coarse_max_dofs=args.coarse_max_dofs, asm_weighting=args.asm_weighting,
                                outer_relax=1 - args.outer_relax)

            def other_relax(s):
                prev_end = sols[s][(nt - 1) * nn:]
                ctxr.rhs(F[s], rhs, u0=prev_end)
                ctxr.guess_previous(prev_end, u)
                return ctxr.solve(rhs, u)
            other_relax(slab_of(args.warmup))
            t_r, o_r = timed(other_relax, min(args.steps, 8))
            compare[f"outer_relax_{1 - args.outer_relax}"] = {
                "value": dofs_per_step * min(args.steps, 8) / (t_r / 1e3), "unit": UNIT,
                "fgmres_iterations_mean": float(np.mean([x["iterations"] for x in o_r]))}
            ctxr.close()

            def weighted(s):
                prev_end = sols[s][(nt - 1) * nn:]
                ctxw.rhs(F[s], rhs, u0=prev_end)
                ctxw.guess_previous(prev_end, u)
                return ctxw.solve(rhs, u)
            weighted(slab_of(args.warmup))
            k4 = min(args.steps, 8)
            t_w, o_w = timed(weighted, k4)
            compare[f"asm_weighting_{other}"] = {"value": dofs_per_step * k4 / (t_w / 1e3), "unit": UNIT,
                                                 "outer_relax": 0,
                                          "fgmres_iterations_mean": float(np.mean([x["iterations"] for x in o_w])),
                                          "omega": [ctxw.level_info(l)["omega"] for l in range(ctxw.n_levels - 1)]}
            ctxw.close()
        if args.atonce_slabs > 1:
            compare["at_once"] = at_once_arm(args, stmg, wl, F, sols, dofs_per_step, nt, nn, inv_prec, dev)

    # end to end through the C ABI from pinned host buffers (H2D of f and the previous slab, D2H of u)
    Fh = torch.empty((n_slabs, n), dtype=torch.float64).pin_memory()
    Fh.copy_(F.cpu())
    Sh = torch.empty((n_slabs + 1, n), dtype=torch.float64).pin_memory()
    Sh.copy_(sols.cpu())
    uh = torch.zeros(n, dtype=torch.float64).pin_memory()
    Fn, Sn, un = Fh.numpy(), Sh.numpy(), uh.numpy()
    e2e_steps = max(1, args.steps)  # the same slabs as the device-timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        s = slab_of(args.warmup + i)
        # the result lands straight in the pinned host state (the next slab's input): no host copy
        if net is not None:
            net.solve_slab_host(Fn[s], Sn[s], Sn[s + 1])
        else:
            ctx.solve_slab_host(Fn[s].reshape(nt, nn), Sn[s][(nt - 1) * nn:], out_u=Sn[s + 1].reshape(nt, nn))
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * dofs_per_step * e2e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": int(8 * (2 * n if net is not None else n + nn)), "d2h_bytes_per_step": int(8 * n)}

    roof, cpu, extra = None, None, {}
    if rank == 0:
        apply_ms = ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.FP64, reps=20)
        asm_ms = ctx.time_kernel(stmg.KERNEL_ASM, 0, stmg.FP32, reps=20)
        inv_bytes = {"fp32": 4, "bf16": 2, "fp64": 8, "fp8": 1}[args.inverse if not args.plain else "fp64"]
        vc_ms = ctx.time_kernel(stmg.KERNEL_VCYCLE, 0, vprec, reps=10)
        nq = wl["p"] + 1
        cells = wl["N"] ** 3
        flops = (12 * nq ** 4 + (16 + 8 * nt) * nq ** 3) * cells * nt
        peaks = read_peaks()
        fp64_peak = 1.25e12
        # double-float: one multiply-add = 15 FP32-pipe instructions (product 4, renormalised sum 11);
        # FP32 pipe = 152 SMs x 128 lanes x 2.07 GHz instructions/s -> FP64-equivalent flop/s peak
        df_peak = 152 * 128 * 2.07e9 / 15 * 2
        roof_fp64 = {"kernel": "apply3d_kernel<N=3,NT=3,double> (finest level, FP64)", "bound": "alu",
                     "achieved": flops / (apply_ms * 1e-3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                     "frac": flops / (apply_ms * 1e-3) / fp64_peak, "traffic": read_traffic("apply_fp64"),
                     "peak_source": "FP64 1.25 TFLOP/s nominal (GB300 table; no measured FP64 peak)",
                     "avg_launch_ms": apply_ms}
        nb = nq ** 3
        eig = args.smoother in ("eig", "eig_tc")
        asm_roof = smoother_roofline(args.inverse, cells, nt, nb, n, asm_ms, peaks,
                                     ("eig_tc_kernel<3,3,3,1> (finest-level additive Schwarz, per-cell "
                                      "eigendecompositions, both products on the tensor cores)")
                                     if args.smoother == "eig_tc" else
                                     (f"eig_apply_kernel<3,3,3,float,{args.inverse}> (finest-level additive Schwarz, "
                                      "per-cell eigendecompositions, TMA-fed)") if eig else
                                     (f"asm_apply_tma_kernel<3,3,3,float,{args.inverse}> (finest-level additive Schwarz, "
                                      "TMA-fed)"),
                                     traffic_key=(f"{args.smoother}_{args.inverse}" if eig else f"asm_{args.inverse}")
                                     if args.inverse in ("bf16", "fp8") else None, eig=eig,
                                     tc=args.smoother == "eig_tc")
        if args.plain:
            roof = roof_fp64
            extra["asm_finest"] = asm_roof
        else:
            df_ms = ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.DF32, reps=20)
            # the dominant kernel of the mixed solver by time share: the finest-level smoother (two sweeps
            # per V-cycle); the double-float apply runs only in the iterations before the relaxed ones
            roof = asm_roof
            extra["apply_df_finest"] = {
                "kernel": "apply3d_kernel<N=3,NT=3,df64,float->double> (finest level, FGMRES apply in double-float)",
                "bound": "alu", "achieved": flops / (df_ms * 1e-3) / 1e12, "peak": df_peak / 1e12, "unit": "TFLOP/s",
                "frac": flops / (df_ms * 1e-3) / df_peak, "traffic": read_traffic("apply_df32"),
                "peak_source": "FP32 pipe 152 x 128 x 2.07 GHz / 15 instructions per double-float multiply-add, "
                               "in FP64-equivalent flop/s (derived)", "avg_launch_ms": df_ms}
            extra["apply_fp64_finest"] = roof_fp64
            f32_ms = ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.FP32, reps=20)
            f32_peak = 152 * 128 * 2 * 2.07e9  # FP32 FMA lanes x 2 flop x max SM clock
            # bytes: x read, y read and written (atomics), the stored FP32 geometry (chunked, 32 B per Gauss point)
            f32_bytes = n * 4 * 3 + cells * nq ** 3 * 32
            extra["apply_fp32_finest"] = {
                "kernel": "apply3d_reg_kernel<3,3,float,float,0> (finest level, V-cycle residuals; one thread per "
                          "cell and time DoF, sum factorisation in registers)", "bound": "alu",
                "achieved": flops / (f32_ms * 1e-3) / 1e12, "peak": f32_peak / 1e12, "unit": "TFLOP/s",
                "frac": flops / (f32_ms * 1e-3) / f32_peak, "avg_launch_ms": f32_ms,
                "stored_bytes": f32_bytes, "hbm_frac": f32_bytes / (f32_ms * 1e-3) / (peaks["hbm_gbs"] * 1e9),
                "traffic": read_traffic("apply_fp32"),
                "note": "frac: of the FP32-pipe peak (algorithmic flop count); hbm_frac: the bytes it must move "
                        "(vectors and the stored geometry) over the measured copy bandwidth; latency-bound "
                        "(long-scoreboard stalls, 16 warps per SM)"}
        extra["vcycle_ms"] = vc_ms
        extra["apply_gdofs"] = apply_gdofs(stmg, ctx, dofs_per_step, df=not args.plain)
        if not args.skip_compare and not args.plain:
            mixed_kw = dict(vcycle_precision=stmg.FP32, inverse_precision=inv_prec, coarse_max_dofs=args.coarse_max_dofs,
                            asm_weighting=args.asm_weighting, outer_relax=args.outer_relax)
            extra["error_vs_fp64"] = {sp_["name"]: slab_error_vs_fp64(stmg, torch, dev, sp_, mixed_kw)
                                      for sp_ in accuracy_specs(stmg)}
            extra["error_vs_fp64"]["definition"] = ("relative L2 difference of the mixed solution (rtol 1e-8) from "
                                                    "the plain FP64 solver's solution of the same slab at rtol 1e-12")
        if not args.skip_cpu:
            r_all = oracle_subprocess(ORACLE_SAMPLE_CELLS, 4, 1, os.cpu_count())
            r_one = oracle_subprocess(ORACLE_SAMPLE_CELLS, 2, 1, 1)
            cpu = {"value": r_all["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "value_1_thread": r_one["value"], "sample": oracle_sample_text(r_all, ORACLE_SAMPLE_CELLS)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.plain else ("f64+df32+f32+bf16" if use_net else "f64+df32+f32"),
            "data": "synthetic",
            "config": {"workload": wl["name"], "cells": wl["N"] ** 3, "p": wl["p"], "time": f"dG({wl['k']})",
                       "dofs_per_step": dofs_per_step, "rtol": 1e-8, "vcycle": "fp64" if args.plain else "fp32",
                       "guess": "learned (fallback previous slab)" if use_net else "previous slab",
                       "schwarz_sum": "weighted by inverse node multiplicity" if args.asm_weighting else
                                      "eq. vanka0 as printed (unweighted)",
                       "dtype_note": f"FP64 FGMRES vectors, dot products and residuals; FGMRES operator apply in double-float "
                                     f"(FP32 pairs) on the FP32 V-cycle outputs; FP32 V-cycle; "
                                     f"{args.inverse.upper()} Schwarz inverses",
                       "slabs_timed": f"{slab_of(args.warmup)}..{slab_of(args.warmup + args.steps - 1)} (held out)"
                       if use_net else "from slab 0",
                       "parallelism": f"replicas{world}", "l2": "working set > L2 (inverses alone 0.15 GB in BF16)",
                       "levels": ctx.n_levels,
                       "coarsest": (f"first level with <= {args.coarse_max_dofs} unknowns, dense inverse"
                                    if args.coarse_max_dofs else "2^3 cells, lowest time degree, dense inverse"),
                       "fgmres_iterations_mean": float(np.mean(its)) if its else None,
                       "relaxed_iterations_mean": float(np.mean(relaxed)) if relaxed else None,
                       "outer_apply": ("double-float; FP32 once the residual estimate is <= 1e5 x the target "
                                       "(inexact Krylov)") if args.outer_relax and not args.plain else
                                      ("FP64" if args.plain else "double-float"),
                       "learned_guess_taken": int(sum(taken)) if use_net else None},
            "gpu_launches": int(launches), "clocks": clk.summary(), "e2e": e2e, "roofline": roof,
            "cpu_baseline": cpu, "kernels": extra, "training": train_info, "compare": compare}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if net is not None:
        net.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def at_once_arm(args, stmg, wl, F, sols, dofs_per_step, nt, nn, inv_prec, dev):
    """The first n_c slabs as one system (eq. heat-cg-dg-at-once) with tau-levels in the hierarchy:
    right-hand side, previous-slab guess and one FGMRES solve to 1e-8 relative residual of the whole
    system, repeated; the solution is compared with the slab-by-slab one of the main arm."""
    import torch
    nc = args.atonce_slabs
    n = nt * nn
    ctxb = stmg.Context(3, wl["N"], wl["p"], wl["k"], wl["tau"], vertices=wl["vertices"], coeff=wl["rho"],
                        vcycle_precision=stmg.FP32, inverse_precision=inv_prec, rtol=1e-8, restart=30, max_it=200,
                        n_slabs=nc, asm_weighting=args.asm_weighting, smoother_kind=smoother_kind(stmg, args))
    rb = torch.empty(nc * n, dtype=torch.float64, device=dev)
    ub = torch.empty_like(rb)
    prev_end = sols[0][(nt - 1) * nn:]

    def once():
        ctxb.rhs(F[:nc].reshape(-1), rb, u0=prev_end)
        ctxb.guess_previous(prev_end, ub)
        return ctxb.solve(rb, ub)
    once()
    reps = 3
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    sts = [once() for _ in range(reps)]
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    seq = sols[1:nc + 1].reshape(-1)
    diff = float((ub - seq).norm() / seq.norm())
    asm_ms = ctxb.time_kernel(stmg.KERNEL_ASM, 0, stmg.FP32, reps=20)
    levels = [ctxb.level_info(l) for l in range(ctxb.n_levels)]
    out = {"slabs_per_system": nc, "value": nc * dofs_per_step / (ms / 1e3), "unit": UNIT, "ms_per_system": ms,
           "fgmres_iterations": sts[-1]["iterations"], "rel_diff_to_slab_by_slab": diff,
           "levels": [f"Q{l['p']} {l['n_cells']}^3 dG({l['k']}) x{l['n_slabs']}" for l in levels],
           "asm_finest_ms_all_slabs": asm_ms, "asm_finest_ms_per_slab": asm_ms / nc}
    ctxb.close()
    return out


def run_learned_c5(args):
    """Learned initial guess vs previous-slab guess on held-out slabs of the moving-Gaussian workload."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N, p, k, n_slabs = args.n_cells if args.n_cells != 32 else 48, 2, 1, 256
    tau = 1.0 / n_slabs
    n_train = n_slabs // 2
    ctx = stmg.Context(3, N, p, k, tau, vcycle_precision=stmg.FP32, rtol=1e-8, restart=30, max_it=200,
                       asm_weighting=args.asm_weighting, outer_relax=args.outer_relax)
    nt, nn = ctx.nt, ctx.n_nodes
    n = nt * nn
    X = ctx.node_coords()
    src = synth.MovingGaussians()
    tn = radau_nodes(k)
    F = torch.empty((n_slabs, n), dtype=torch.float64, device=dev)
    for s_ in range(n_slabs):
        F[s_].copy_(torch.from_numpy(np.stack([src(X, tau * (s_ + th)) for th in tn]).reshape(-1)))
    sols = torch.zeros((n_slabs + 1, n), dtype=torch.float64, device=dev)
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    cand = torch.empty(n, dtype=torch.float64, device=dev)
    dofs = nt * (N * p - 1) ** 3

    def slab(s_, net=None):
        prev = sols[s_]
        prev_end = prev[(nt - 1) * nn:]
        ctx.rhs(F[s_], rhs, u0=prev_end)
        ctx.guess_previous(prev_end, u)
        taken = False
        if net is not None:
            net.predict(prev, F[s_], cand)
            taken = ctx.select_guess(rhs, cand, u)
        st = ctx.solve(rhs, u)
        assert st["converged"], st
        sols[s_ + 1].copy_(u)
        return st, taken

    t0 = time.perf_counter()
    for s_ in range(n_train):
        slab(s_)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    su = 1.0 / float(sols[1:n_train + 1].pow(2).mean().sqrt())
    sf = 1.0 / float(F[:n_train].pow(2).mean().sqrt())
    incr = torch.stack([sols[s_ + 1] - sols[s_][(nt - 1) * nn:].repeat(nt) for s_ in range(1, n_train)])
    so = 1.0 / float(incr.pow(2).mean().sqrt())
    channels = (2 * nt, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, NET_CHANNELS_HIDDEN, nt)
    W, b = synth.conv_net_init(channels, seed=15)
    net = stmg.Net(ctx, channels, W, b, (su, sf, so))
    t1 = time.perf_counter()
    losses = []
    order = np.random.default_rng(16).permutation
    for epoch in range(args.epochs):
        for s_ in order(np.arange(1, n_train)):
            losses.append(net.train_step(sols[s_], F[s_], sols[s_ + 1], args.lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    ref_sols = sols.clone()
    arms = {}
    for name, use in (("learned", True), ("previous_slab", False)):
        sols.copy_(ref_sols)
        its, taken = [], []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for s_ in range(n_train, n_slabs):
            st, tk = slab(s_, net if use else None)
            its.append(st["iterations"])
            taken.append(tk)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        arms[name] = {"value": dofs * (n_slabs - n_train) / (ms / 1e3), "unit": UNIT, "ms_per_slab": ms / (n_slabs - n_train),
                      "fgmres_iterations_mean": float(np.mean(its)), "guess_taken": int(sum(taken))}
    # the plain FP64 solver (FP64 V-cycle, FP64 operator apply) on the first held-out slabs, previous-slab guess
    ctx64 = stmg.Context(3, N, p, k, tau, vcycle_precision=stmg.FP64, rtol=1e-8, restart=30, max_it=200,
                         asm_weighting=args.asm_weighting)
    sols.copy_(ref_sols)
    n64 = min(16, n_slabs - n_train)
    its64 = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for s_ in range(n_train, n_train + n64):
        prev_end = sols[s_][(nt - 1) * nn:]
        ctx64.rhs(F[s_], rhs, u0=prev_end)
        ctx64.guess_previous(prev_end, u)
        st = ctx64.solve(rhs, u)
        assert st["converged"], st
        sols[s_ + 1].copy_(u)
        its64.append(st["iterations"])
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    arms["plain_fp64_previous_slab"] = {"value": dofs * n64 / (ms64 / 1e3), "unit": UNIT, "ms_per_slab": ms64 / n64,
                                        "fgmres_iterations_mean": float(np.mean(its64)),
                                        "slabs": f"{n_train}..{n_train + n64 - 1}"}
    ctx64.close()
    pred_ms = []
    for _ in range(10):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record()
        net.predict(sols[n_train], F[n_train], cand)
        b_.record()
        torch.cuda.synchronize()
        pred_ms.append(a_.elapsed_time(b_))
    voxels = (N * p + 1) ** 3
    conv_flops = 2 * 27 * voxels * sum(channels[l] * channels[l + 1] for l in range(len(channels) - 1))
    inference = {"median_ms": float(np.median(pred_ms)), "flops": conv_flops,
                 "tflops": conv_flops / (float(np.median(pred_ms)) * 1e-3) / 1e12,
                 "frac_of_bf16_burst": conv_flops / (float(np.median(pred_ms)) * 1e-3) / 1e12 /
                 read_peaks()["bf16_tflops"]}
    line = {"metric": "space-time DoFs/s solved to 1e-8, learned vs previous-slab initial guess (held-out slabs)",
            "value": arms["learned"]["value"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": f"heat3d_q2_dg1_{N}cubed_8movinggaussians", "slabs": n_slabs, "train_slabs": n_train,
                       "eval_slabs": f"{n_train}..{n_slabs - 1}", "dofs_per_slab": dofs, "epochs": args.epochs,
                       "lr": args.lr, "channels": list(channels)},
            "training": {"data_solve_s": t_data, "train_s": t_train, "steps": len(losses),
                         "loss_first_epoch": float(np.mean(losses[:n_train - 1])),
                         "loss_last_epoch": float(np.mean(losses[-(n_train - 1):]))},
            "inference": inference, "arms": arms}
    print(json.dumps(line), flush=True)
    net.close()
    ctx.close()
    return 0


def run_c4(args):
    """Config 4: heat, Q4 on 64^3 Cartesian cells, dG(3), smooth coefficient at the Gauss points,
    fast-diagonalisation local solves; mixed (FP32 V-cycle) and plain FP64 solvers, 8 slabs."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N = args.n_cells if args.n_cells != 32 else 64
    p, k, n_slabs = 4, 3, 8
    tau = 1.0 / n_slabs
    V = synth.cartesian_vertices(N, 3)
    a, phi = synth.smooth_coefficient_params(3)
    # the coefficient is evaluated at the Gauss points of the Cartesian cells
    xq = np.polynomial.legendre.leggauss(p + 1)[0] * 0.5 + 0.5
    ql = np.indices((p + 1,) * 3).reshape(3, -1)[::-1].T
    cells = np.indices((N,) * 3).reshape(3, -1)[::-1].T
    pts = (cells[:, None, :] + xq[ql][None, :, :]) / N
    rho_qp = synth.smooth_coefficient_at(pts, a, phi)
    out = {}
    tn = radau_nodes(k)
    for name, prec in (("mixed_fp32_vcycle", stmg.FP32), ("plain_fp64", stmg.FP64)):
        t0 = time.perf_counter()
        ctx = stmg.Context(3, N, p, k, tau, vertices=None, coeff=rho_qp.reshape(-1), coeff_mode=stmg.COEFF_PER_QPOINT,
                           vcycle_precision=prec, rtol=1e-8, restart=30, max_it=200, asm_weighting=args.asm_weighting)
        t_setup = time.perf_counter() - t0
        nt, nn = ctx.nt, ctx.n_nodes
        X = ctx.node_coords()
        rhs = torch.empty(nt * nn, dtype=torch.float64, device=dev)
        u = torch.empty_like(rhs)
        u_prev = torch.zeros(nn, dtype=torch.float64, device=dev)
        steps = n_slabs if prec == stmg.FP32 else min(2, n_slabs)
        its = []
        ms = 0.0
        for s_ in range(steps):
            f = torch.from_numpy(np.stack([synth.heat_sine_source(X, tau * (s_ + th)) for th in tn]).reshape(-1)).to(dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.rhs(f, rhs, u0=u_prev)
            ctx.guess_previous(u_prev, u)
            st = ctx.solve(rhs, u)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            assert st["converged"], st
            its.append(st["iterations"])
            u_prev.copy_(u[(nt - 1) * nn:])
        dofs = nt * (N * p - 1) ** 3
        out[name] = {"value": dofs * steps / (ms / 1e3), "unit": UNIT, "ms_per_slab": ms / steps,
                     "fgmres_iterations_mean": float(np.mean(its)), "slabs": steps, "setup_s": t_setup,
                     "apply_fp64_ms": ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.FP64, reps=5),
                     "apply_fp32_ms": ctx.time_kernel(stmg.KERNEL_APPLY, 0, stmg.FP32, reps=5),
                     "fd_smoother_fp32_ms": ctx.time_kernel(stmg.KERNEL_ASM, 0, stmg.FP32, reps=5),
                     "vcycle_ms": ctx.time_kernel(stmg.KERNEL_VCYCLE, 0, prec, reps=3)}
        ctx.close()
    line = {"metric": "space-time DoFs/s solved to 1e-8 rel. residual", "value": out["mixed_fp32_vcycle"]["value"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"heat3d_q4_dg3_{N}cubed_cartesian_smoothrho", "dofs_per_slab": nt * (N * p - 1) ** 3,
                       "smoother": "fast diagonalisation (cell-mean coefficient)"},
            "arms": out}
    print(json.dumps(line), flush=True)
    return 0


def run_c3(args):
    """Wave workload: first-order-in-time acoustic wave condensed to the displacement, Q3 on 24^3 cells
    with interior vertices jittered by U[-0.15h, 0.15h], cGP(2), tau = 1/64 (64 slabs), rho = c^2 = 1
    below z = 0.5 and 16 above (c = 1 / 4), Gaussian pulse u0 (sigma 0.05 at (0.5, 0.5, 0.25)), v0 = 0,
    f = 0.  One step = one slab: right-hand side, previous-slab guess, FGMRES with the FP32 V-cycle to
    rtol 1e-8, velocity update."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N, p, k, n_slabs = 24, 3, 2, 64
    tau = 1.0 / n_slabs
    V = synth.jittered_vertices(N, 3)
    rho = synth.layer_coefficient(N, 3, 1.0, 16.0)
    inv_prec = {"fp32": stmg.FP32, "bf16": stmg.BF16, "fp64": stmg.FP64, "fp8": stmg.FP8}[args.inverse]
    t0 = time.perf_counter()
    ctx = stmg.Context(3, N, p, k, tau, pde=stmg.WAVE, scheme=stmg.CGP, vertices=V, coeff=rho,
                       vcycle_precision=stmg.FP32, inverse_precision=inv_prec, rtol=1e-8, restart=30, max_it=200,
                       coarse_max_dofs=args.coarse_max_dofs, asm_weighting=args.asm_weighting,
                       outer_relax=args.outer_relax, smoother_kind=smoother_kind(stmg, args))
    setup_s = time.perf_counter() - t0
    nt, nn = ctx.nt, ctx.n_nodes
    n = nt * nn
    X = ctx.node_coords()
    bnd = np.any((X < 1e-12) | (X > 1.0 - 1e-12), axis=1)
    u0 = synth.wave_pulse(X)
    u0[bnd] = 0.0
    dofs = nt * (N * p - 1) ** 3
    zf = torch.zeros(n, dtype=torch.float64, device=dev)
    zn = torch.zeros(nn, dtype=torch.float64, device=dev)
    rhs = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    v = torch.empty(n, dtype=torch.float64, device=dev)
    u_prev = torch.from_numpy(u0).to(dev)
    v_prev = torch.zeros(nn, dtype=torch.float64, device=dev)

    def step():
        ctx.rhs(zf, rhs, f0=zn, u0=u_prev, v0=v_prev)
        ctx.guess_previous(u_prev, u)
        st = ctx.solve(rhs, u)
        if not st["converged"]:
            raise RuntimeError(f"wave slab did not converge: {st}")
        ctx.wave_velocity(u, u_prev, v_prev, v)
        u_prev.copy_(u[(nt - 1) * nn:])
        v_prev.copy_(v[(nt - 1) * nn:])
        return st

    steps = min(args.steps, n_slabs - args.warmup)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    its, relaxed = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            st = step()
            its.append(st["iterations"])
            relaxed.append(st["relaxed_iterations"])
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    peaks = read_peaks()
    asm_ms = ctx.time_kernel(stmg.KERNEL_ASM, 0, stmg.FP32, reps=20)
    cells, nq = N ** 3, p + 1
    roof = smoother_roofline(args.inverse, cells, nt, nq ** 3, n, asm_ms, peaks,
                             f"{'eig_apply_kernel' if args.smoother == 'eig' else 'asm_apply_tma_kernel'}"
                             f"<3,4,2,float,{args.inverse}> (finest-level additive Schwarz)",
                             eig=args.smoother in ("eig", "eig_tc"), tc=args.smoother == "eig_tc")
    ga = apply_gdofs(stmg, ctx, dofs)
    flops = (12 * nq ** 4 + (16 + 8 * nt) * nq ** 3) * cells * nt
    df_peak = 152 * 128 * 2.07e9 / 15 * 2
    f32_peak = 152 * 128 * 2 * 2.07e9
    kernels = {
        "apply_gdofs": ga,
        "apply_df_finest": {"bound": "alu", "achieved": flops / (ga["df32"]["median_ms"] * 1e-3) / 1e12,
                            "peak": df_peak / 1e12, "unit": "TFLOP/s",
                            "frac": flops / (ga["df32"]["median_ms"] * 1e-3) / df_peak},
        "apply_fp32_finest": {"bound": "alu", "achieved": flops / (ga["fp32"]["median_ms"] * 1e-3) / 1e12,
                              "peak": f32_peak / 1e12, "unit": "TFLOP/s",
                              "frac": flops / (ga["fp32"]["median_ms"] * 1e-3) / f32_peak},
        "vcycle_ms": ctx.time_kernel(stmg.KERNEL_VCYCLE, 0, stmg.FP32, reps=10)}
    levels = [ctx.level_info(l) for l in range(ctx.n_levels)]
    ctx.close()
    err = None
    if not args.skip_compare:
        mixed_kw = dict(vcycle_precision=stmg.FP32, inverse_precision=inv_prec, coarse_max_dofs=args.coarse_max_dofs,
                        asm_weighting=args.asm_weighting, outer_relax=args.outer_relax)
        err = slab_error_vs_fp64(stmg, torch, dev, accuracy_specs(stmg)[2], mixed_kw)
    line = {"metric": "space-time DoFs/s solved to 1e-8 rel. residual (mixed FP32 V-cycle in FP64 FGMRES)",
            "value": dofs * steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms / steps, "higher_is_better": True, "dtype": "f64+df32+f32", "data": "synthetic",
            "config": {"workload": C3_NAME, "cells": cells, "p": p, "time": "cGP(2)", "dofs_per_step": dofs,
                       "slabs_timed": f"{args.warmup}..{args.warmup + steps - 1}", "rtol": 1e-8,
                       "levels": [f"Q{l['p']} {l['n_cells']}^3 cGP({l['k']})" for l in levels],
                       "inverse_storage": args.inverse, "setup_s": setup_s,
                       "fgmres_iterations_mean": float(np.mean(its)),
                       "relaxed_iterations_mean": float(np.mean(relaxed)),
                       "schwarz_sum": "weighted by inverse node multiplicity" if args.asm_weighting else
                                      "eq. vanka0 as printed (unweighted)"},
            "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof, "kernels": kernels,
            "error_vs_fp64": err}
    print(json.dumps(line), flush=True)
    return 0


def run_shm(args):
    """Structural-health-monitoring-like wave problem (Section 4.3), reduced: [-1, 1]^3 on N^3 Cartesian
    cells (N a multiple of 5), Q2, cGP(2), highly heterogeneous coefficient (layers 1 / 9 / 16 times
    c ~ U[0.4, 1.6] per cell of the 5^3 coarse grid), bump initial displacement (radius s = 4h instead
    of 0.01: resolvable on the reduced grid), v = 0, f = 0, tau = 2 / (5 * 2^(r+1)) with N = 5 * 2^r.
    Slab by slab for nu = 1, 2, 4 smoothing steps (the paper's table iter-wave-hc), point values at
    the three goal points every slab."""
    import torch
    import paper_2408_04372_gb300 as stmg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N = args.n_cells if args.n_cells != 32 else 40
    r = int(round(np.log2(N / 5)))
    p, k = 2, 2
    tau = 2.0 / (5 * 2 ** (r + 1))
    V = synth.cartesian_vertices(N, 3, lo=-1.0, hi=1.0)
    rho = synth.shm_coefficient(N, rough=True)
    steps = max(args.steps, 3)
    out = {}
    for nu in (1, 2, 4):
        ctx = stmg.Context(3, N, p, k, tau, pde=stmg.WAVE, scheme=stmg.CGP, vertices=V, coeff=rho,
                           nu_pre=nu, nu_post=nu, vcycle_precision=stmg.FP32, inverse_precision=stmg.BF16, rtol=1e-8,
                           restart=30, max_it=200, coarse_max_dofs=args.coarse_max_dofs,
                           asm_weighting=args.asm_weighting)
        nt, nn = ctx.nt, ctx.n_nodes
        X = ctx.node_coords()
        u0 = synth.shm_initial(X, s=4.0 * 2.0 / N)
        u0[np.any(np.abs(np.abs(X) - 1.0) < 1e-12, axis=1)] = 0.0
        rhs = torch.empty(nt * nn, dtype=torch.float64, device=dev)
        u = torch.empty_like(rhs)
        v = torch.empty_like(rhs)
        zf = torch.zeros(nt * nn, dtype=torch.float64, device=dev)
        zn = torch.zeros(nn, dtype=torch.float64, device=dev)
        u_prev = torch.from_numpy(u0).to(dev)
        v_prev = torch.zeros(nn, dtype=torch.float64, device=dev)
        its, goal, ms = [], [], 0.0
        for s_ in range(args.warmup + steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.rhs(zf, rhs, f0=zn, u0=u_prev, v0=v_prev)
            ctx.guess_previous(u_prev, u)
            st = ctx.solve(rhs, u)
            ctx.wave_velocity(u, u_prev, v_prev, v)
            e1.record()
            torch.cuda.synchronize()
            assert st["converged"], st
            if s_ >= args.warmup:
                ms += e0.elapsed_time(e1)
                its.append(st["iterations"])
            goal.append(ctx.point_values(u, synth.SHM_POINTS)[:, -1].tolist())
            u_prev.copy_(u[(nt - 1) * nn:])
            v_prev.copy_(v[(nt - 1) * nn:])
        dofs = nt * (N * p - 1) ** 3
        out[f"nu_{nu}"] = {"value": dofs * steps / (ms / 1e3), "unit": UNIT, "ms_per_slab": ms / steps,
                           "fgmres_iterations_mean": float(np.mean(its)), "slabs_timed": steps,
                           "goal_point_values_at_slab_ends": goal}
        ctx.close()
    line = {"metric": "space-time DoFs/s solved to 1e-8 rel. residual", "value": out["nu_1"]["value"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f64+df32+f32", "data": "synthetic",
            "config": {"workload": f"wave3d_q2_cgp2_{N}cubed_shm_rough", "dofs_per_slab": 2 * (N * p - 1) ** 3,
                       "tau": tau, "goal_points": list(synth.SHM_POINTS)},
            "arms": out}
    print(json.dumps(line), flush=True)
    return 0


def smoother_kind(stmg, args):
    return {"auto": stmg.SMOOTHER_AUTO, "dense": stmg.SMOOTHER_DENSE, "eig": stmg.SMOOTHER_EIG,
            "eig_tc": stmg.SMOOTHER_EIG_TC}[args.smoother]


def smoother_roofline(inverse, cells, nt, nb, n, asm_ms, peaks, kernel_name, traffic_key=None, eig=False, tc=False):
    """Finest-level Schwarz sweep against the measured copy bandwidth.  Algorithmic bytes: the
    stored local solver without padding -- n_b^2 inverse entries per time plane and cell, or with the
    eigendecomposition smoother the n_b^2 entries of Q and n_b FP32 eigenvalues per cell -- plus two
    FP32 vectors (residual in, correction out); the stored block with its padding is reported apart."""
    inv_bytes = {"fp32": 4, "bf16": 2, "fp64": 8, "fp8": 1}[inverse]
    nbp = (nb + 3) // 4 * 4
    if tc:
        nq = 16 if nb <= 16 else 32 if nb <= 32 else 64  # BF16 operand images padded to nq x nq
        alg = cells * (nb * nb * 2 + 4 * nb) + 2 * 4 * n
        stored = cells * (nq * nq * 2 + 4 * nq) + 2 * 4 * n
    elif eig:
        inv_bytes = 2 if inverse == "fp8" else inv_bytes  # FP8 requests store Q in BF16
        mu_bytes = 8 if inv_bytes == 8 else 4
        nbq = nbp if (nbp // 4) % 2 == 1 else nbp + 4  # Q's row stride (odd number of 4-entry chunks)
        alg = cells * (nb * nb * inv_bytes + mu_bytes * nb) + 2 * 4 * n
        stored = cells * ((nb * nbq * inv_bytes + mu_bytes * nbq + 15) // 16 * 16) + 2 * 4 * n
    else:
        alg = cells * nt * nb * nb * inv_bytes + 2 * 4 * n
        plane_entries = nt * nb * nbp
        cell_bytes = ((plane_entries + 4 * nt + 15) // 16 * 16 if inv_bytes == 1 else
                      (plane_entries + 7) // 8 * 8 * inv_bytes)
        stored = cells * cell_bytes + 2 * 4 * n
    gbs = alg / (asm_ms * 1e-3) / 1e9
    return {"kernel": kernel_name, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"],
            "traffic": read_traffic(traffic_key) if traffic_key else None,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured",
            "algorithmic_bytes": alg, "stored_bytes_with_padding": stored, "inverse_storage": inverse,
            "avg_launch_ms": asm_ms}


def median_launch_ms(ctx, kind, level, prec, warm=10, reps=100):
    """Median of `reps` single-launch CUDA-event timings after `warm` launches (each timing brackets one
    launch on the context's stream)."""
    for _ in range(warm):
        ctx.time_kernel(kind, level, prec, reps=1)
    return float(np.median([ctx.time_kernel(kind, level, prec, reps=1) for _ in range(reps)]))


def apply_gdofs(stmg, ctx, dofs, df=True):
    """Operator apply throughput on the finest level: N_t x interior nodes / median launch time."""
    out = {}
    precs = [("fp64", stmg.FP64), ("fp32", stmg.FP32)] + ([("df32", stmg.DF32)] if df else [])
    for name, prec in precs:
        ms = median_launch_ms(ctx, stmg.KERNEL_APPLY, 0, prec)
        out[name] = {"gdofs": dofs / (ms * 1e-3) / 1e9, "median_ms": ms}
    out["definition"] = "N_t x interior nodes / median of 100 single-launch CUDA-event timings after 10 warm-up"
    return out


def slab_error_vs_fp64(stmg, torch, dev, spec, mixed_kw):
    """Relative L2 difference between the mixed solver's slab solution (rtol 1e-8, the bench's options)
    and the plain FP64 solver's solution of the same slab from the same guess at rtol 1e-12."""
    dim, N, p, k, pde, scheme, tau, V, rho, slab_index = (spec[x] for x in (
        "dim", "N", "p", "k", "pde", "scheme", "tau", "vertices", "rho", "slab"))
    sols = {}
    for name, kw in (("mixed", dict(mixed_kw, rtol=1e-8)),
                     ("fp64", dict(vcycle_precision=stmg.FP64, rtol=1e-12, coarse_max_dofs=mixed_kw.get("coarse_max_dofs", 0),
                                   asm_weighting=mixed_kw.get("asm_weighting", 0)))):
        ctx = stmg.Context(dim, N, p, k, tau, pde=pde, scheme=scheme, vertices=V, coeff=rho, restart=30, max_it=400, **kw)
        nt, nn = ctx.nt, ctx.n_nodes
        X = ctx.node_coords()
        bnd = np.any((X < 1e-12) | (X > 1.0 - 1e-12), axis=1)
        rhs = torch.empty(nt * nn, dtype=torch.float64, device=dev)
        u = torch.empty_like(rhs)
        t0 = tau * slab_index
        if pde == stmg.HEAT:
            tn = radau_nodes(k) if scheme == stmg.DG else np.linspace(0.0, 1.0, k + 1)[1:]
            f = np.stack([synth.heat_sine_source(X, t0 + tau * th) for th in tn])
            u0 = synth.heat_sine_solution(X, t0)
            u0[bnd] = 0.0
            u0d = torch.from_numpy(u0).to(dev)
            ctx.rhs(torch.from_numpy(f.reshape(-1)).to(dev), rhs, u0=u0d)
        else:
            u0 = synth.wave_pulse(X)
            u0[bnd] = 0.0
            u0d = torch.from_numpy(u0).to(dev)
            ctx.rhs(torch.zeros(nt * nn, dtype=torch.float64, device=dev), rhs,
                    f0=torch.zeros(nn, dtype=torch.float64, device=dev), u0=u0d,
                    v0=torch.zeros(nn, dtype=torch.float64, device=dev))
        ctx.guess_previous(u0d, u)
        st = ctx.solve(rhs, u)
        if not st["converged"]:
            raise RuntimeError(f"{spec['name']} {name} did not converge: {st}")
        sols[name] = (u.clone(), st)
        ctx.close()
    um, ur = sols["mixed"][0], sols["fp64"][0]
    return {"rel_l2_error": float((um - ur).norm() / ur.norm()), "mixed_iterations": sols["mixed"][1]["iterations"],
            "fp64_iterations_rtol_1e-12": sols["fp64"][1]["iterations"], "slab": slab_index}


def accuracy_specs(stmg):
    """One slab of each of the three solved configurations: 2D heat (Q2 16^2, dG(1)), the headline 3D
    heat workload, and the 3D wave workload (Q3 24^3 jittered, cGP(2), two layers, Gaussian pulse)."""
    return [
        dict(name="c1_heat2d_q2_dg1_16sq", dim=2, N=16, p=2, k=1, pde=stmg.HEAT, scheme=stmg.DG, tau=1 / 16,
             vertices=None, rho=None, slab=1),
        dict(name=workload()["name"], dim=3, N=32, p=2, k=2, pde=stmg.HEAT, scheme=stmg.DG, tau=1 / 32,
             vertices=synth.jittered_vertices(32, 3), rho=synth.block_coefficient(32, 3, blocks=4), slab=3),
        dict(name=C3_NAME, dim=3, N=24, p=3, k=2, pde=stmg.WAVE, scheme=stmg.CGP, tau=1 / 64,
             vertices=synth.jittered_vertices(24, 3), rho=synth.layer_coefficient(24, 3, 1.0, 16.0), slab=0),
    ]


C3_NAME = "wave3d_q3_cgp2_24cubed_jitter0.15_layers1_16_pulse"


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


def source_sha(paths):
    """First 16 hex digits of the SHA-256 over the given source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(key):
    """DRAM bytes per launch from the committed ncu capture; None once a source of the kernel changed."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(key)
    if d is None:
        return None
    srcs = d["sources"] if "sources" in d else [d["source"]]
    if source_sha(srcs) != d["source_sha"]:
        return None
    return d.get("bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-cells", type=int, default=32)
    ap.add_argument("--plain", action="store_true", help="FP64 V-cycle (plain STMG) instead of mixed precision")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-compare", action="store_true", help="skip the no-network and plain-FP64 comparison arms")
    ap.add_argument("--net", action="store_true", help="learned guess on this workload too (trained on slabs 0-15)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "shm", "oracle_c2"])
    ap.add_argument("--oracle-run", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--inverse", default="bf16", choices=["fp32", "bf16", "fp64", "fp8"],
                    help="storage of the Schwarz inverses in the mixed solver")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--smoother", default="dense", choices=["auto", "dense", "eig", "eig_tc"],
                    help="local solver of the Schwarz smoother: stored inverse planes (dense) or per-cell "
                         "eigendecompositions (eig)")
    ap.add_argument("--only-kernel", default=None,
                    choices=["apply64", "apply32", "applydf", "asm32", "asm64", "vcycle32", "vcycle64", "ortho64", "orthodf", "net"],
                    help="profiling helper: time one kernel only (fixed omega, no Arnoldi)")
    ap.add_argument("--level", type=int, default=0,
                    help="multigrid level of --only-kernel (0 = finest); for ortho64 and orthodf the basis size")
    ap.add_argument("--asm-weighting", type=int, default=1, choices=[0, 1],
                    help="1: each cell's Schwarz correction divided by the node's cell count (reading of the "
                         "paper's omega range and iteration tables); 0: the sum of eq. vanka0 as printed")
    ap.add_argument("--outer-relax", type=int, default=1, choices=[0, 1],
                    help="1: FGMRES apply in FP32 once the residual estimate is <= 1e5 x the target (inexact Krylov)")
    ap.add_argument("--atonce-slabs", type=int, default=8,
                    help="comparison arm: the first n slabs as one system with tau-multigrid (0 = off)")
    ap.add_argument("--coarse-max-dofs", type=int, default=1500,
                    help="hierarchy ends at the first coarser level with at most this many unknowns (0: full)")
    args = ap.parse_args()
    if args.oracle_run:
        print(json.dumps(oracle_c2_run(args.oracle_run, args.steps, args.warmup)), flush=True)
        return 0
    if args.only_kernel:
        return run_kernel_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_learned_c5(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "c3":
        return run_c3(args)
    if args.workload == "oracle_c2":
        return run_oracle_full(args)
    if args.workload == "shm":
        return run_shm(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
