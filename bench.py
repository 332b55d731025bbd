"""Benchmark: ms per pressure solve to 1e-8 relative residual at C192L70 on GB300.

One step = one pressure solve H x = b (Eq. helmholtz) by FP64 GCR(5) right-preconditioned
with one multigrid V-cycle per iteration (Algorithm 1, FP32 vectors and coefficients,
FP32 accumulation), from x = 0 to ||b - H x|| <= 1e-8 ||b||, on the synthetic C192L70
workload (221,184 columns x 70 levels = 15,482,880 unknowns, seeded inputs).

Printed JSON line (rank 0):
  value        ms per solve, inputs resident in HBM (whole job: timed region / solves done)
  e2e          the same through the public API with host (pinned) buffers: H2D of b, the
               solve, D2H of x inside every timed step
  roofline     dominant kernel (finest-level block-Jacobi sweep): algorithmic bytes per launch
               / event-timed launch duration, against the measured HBM copy bandwidth
  cpu_baseline the CPU oracle (numpy FP64, as it stands) timed on a bounded sample
  clocks       nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle (the reference of this build) on the same workload:
one GCR iteration of the oracle's pressure solve per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

METRIC = "ms per pressure solve to 1e-8 rel. residual at C192L70"
# Stopping tolerance of the timed solve on the relative residual: at 1e-8 itself the C192L70
# solution's relative error against the oracle's is 1.3e-8 (9 iterations, residual 2.6e-9);
# 2e-9 takes one more iteration and keeps the error below 1e-8 (tests/test_gpu_fullsize.py)
SOLVE_TOL = 2e-9
UNIT = "ms"
WORKLOAD = ("C192L70 pressure solve: GCR(5) FP64 outer + 4-level FP32 V-cycle, stopped at relative residual 2e-9 "
            "(solution error vs the FP64 oracle <= 1e-8)")


SWEEP_VARIANTS = ("plain", "zero", "prolong", "prolong0")


KERNEL_SOURCES = ("kernels.cuh", "krylov.cuh", "mgsolve.cu")   # device code and launch configurations


def _source_digest() -> str:
    """sha256 of the device-code sources: a committed ncu record is used only while it matches."""
    import hashlib
    hsh = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_00756_gb300", "csrc")
    for f in KERNEL_SOURCES:
        hsh.update(open(os.path.join(csrc, f), "rb").read())
    return hsh.hexdigest()


def profiled_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes (read + write) per launch from profiles/dram_traffic.json, if that record
    was taken on the current kernel sources, else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != _source_digest():
        return None
    rec = d.get("kernels", {}).get(f"{workload}/{precision}/{kernel}")
    return None if rec is None else float(rec["dram_bytes_per_launch"])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.result = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            self.result = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                           "samples": len(sm)}


def workload_name(cfg, precision: str) -> str:
    """The headline workload's name, with what differs from it spelled out."""
    name = WORKLOAD if precision == "fp32" else WORKLOAD.replace("FP32", precision)
    if cfg.levels != 4:
        name = name.replace("4-level", f"{cfg.levels}-level")
    if cfg.dt != 600.0:
        name += f", dt {cfg.dt:g} s"
    if cfg.name != "c192":
        name = name.replace("C192L70", f"C{cfg.n}L{cfg.nlev}")
    return name


def max_over_ranks(x: float, pg, device: str) -> float:
    """The maximum of x over all ranks (x itself without a process group): the job's time is
    the slowest replica's."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_unit(ms_max: float, units_per_rank: int, world: int) -> float:
    """Whole-job time per unit: every rank solves `units_per_rank` independent problems (weak
    scaling, replicas), so the job processes units_per_rank * world of them in ms_max."""
    return ms_max / (units_per_rank * world)


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_iteration_time(cfg, inp, iters: int = 1):
    """Seconds per GCR iteration of the oracle's pressure solve (setup excluded)."""
    from oracle.krylov import gcr
    from oracle.problem import pressure_hierarchy
    hier = pressure_hierarchy(cfg, inp)
    H = hier.levels[0]
    P = hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse)
    t0 = time.perf_counter()
    _, it, hist = gcr(H.apply, inp["rhs"], P, tol=0.0, restart=cfg.gcr_restart, maxiter=iters)
    return (time.perf_counter() - t0) / it, hist


def oracle_full_solve(name: str, tol: float):
    """One complete oracle pressure solve of workload `name` from x = 0 to `tol` (FP64 V-cycle
    inside GCR, numpy, one thread): (seconds of the solve, seconds of the set-up, iterations)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle.krylov import gcr
    from oracle.problem import pressure_hierarchy
    cfg = syn.config(name)
    inp = syn.make_inputs(cfg, mixed=False)
    t0 = time.perf_counter()
    hier = pressure_hierarchy(cfg, inp)
    t1 = time.perf_counter()
    P = hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse)
    _, it, hist = gcr(hier.levels[0].apply, inp["rhs"], P, tol=tol, restart=cfg.gcr_restart, maxiter=200)
    return time.perf_counter() - t1, t1 - t0, it


def cpu_baseline_full(tol: float):
    """The oracle's complete solves on the host: C192L70 (the headline workload) once on one
    core, and the smaller workloads C12L30, C48L30 and C96L70 on one core and on all cores at once (one
    process per core, each solving the same problem: whole-host throughput)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    out = {}
    sec, setup, it = oracle_full_solve("c192", tol)
    out["c192"] = {"ms_per_solve_1core": round(sec * 1e3, 1), "setup_s": round(setup, 1), "iters": it}
    ctx = mp.get_context("spawn")
    for name in ("c12", "c48", "c96"):
        s1, _, it1 = oracle_full_solve(name, tol)
        with ctx.Pool(cores) as pool:
            t0 = time.perf_counter()
            res = pool.starmap(oracle_full_solve, [(name, tol)] * cores)
            wall = time.perf_counter() - t0
        # the pool's wall time includes each worker's set-up: take the solves' own times
        solve_max = max(r[0] for r in res)
        out[name] = {"ms_per_solve_1core": round(s1 * 1e3, 1), "iters": it1,
                     "ms_per_solve_all_cores": round(solve_max * 1e3 / cores, 1),
                     "all_cores_wall_s": round(wall, 1)}
    return out, cores


def run_reference(args, cfg, inp, world, rank):
    """CPU oracle arm: one oracle GCR iteration per step, solves restarted from x = 0."""
    if rank != 0:
        return
    from oracle.problem import pressure_hierarchy
    hier = pressure_hierarchy(cfg, inp)
    H = hier.levels[0]
    P = hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse)
    from oracle.krylov import GCR
    b = inp["rhs"]
    for _ in range(args.warmup):          # warm-up: one operator application each
        H.apply(b)
    Solve = lambda: GCR(H.apply, b, P, cfg.gcr_restart)

    s = Solve()
    its, times, per_solve_iters = 0, [], []
    budget_s = 150.0       # the timed steps stop once this much CPU time is spent
    t_start = time.perf_counter()
    for _ in range(args.steps):
        if times and time.perf_counter() - t_start > budget_s:
            break
        t0 = time.perf_counter()
        rel = s.step()
        times.append(time.perf_counter() - t0)
        its += 1
        if rel <= args.tol:
            per_solve_iters.append(its)
            its = 0
            s = Solve()
    sec_it = float(np.mean(times))
    if per_solve_iters:
        n_it = float(np.mean(per_solve_iters))
        how = f"{len(per_solve_iters)} oracle solve(s) completed within the timed steps"
    else:   # extrapolate the observed residual contraction to 1e-8
        rho = rel ** (1.0 / its)
        n_it = float(np.ceil(np.log(args.tol) / np.log(rho)))
        how = f"iterations to 1e-8 extrapolated from {its} steps (mean contraction {rho:.3f})"
    value = sec_it * n_it * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec_it * 1e3, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD.replace("FP32 V-cycle", "FP64 V-cycle (CPU oracle)"),
                                        "n": cfg.n, "nlev": cfg.nlev, "levels": cfg.levels},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one numpy FP64 GCR iteration of the C192L70 solve per step, "
                                   f"{len(times)} steps timed (150 s budget); ms/solve = mean iteration "
                                   f"time x {n_it:.1f} iterations ({how})"},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args, cfg, inp, mg, torch, world, rank):
    """The differentiable solve: forward x = H^-1 b and backward dL/db = H^-T dL/dx through the
    torch autograd wrapper, L = <w, x> (C96L70 by default)."""
    h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=False)
    b0 = torch.from_numpy(inp["rhs"]).cuda()
    wv = torch.from_numpy(syn.normal(cfg.seed, 99, cfg.ncell)).cuda()

    def step():
        b = b0.clone().requires_grad_(True)
        x = mg.solve(h, b, tol=args.tol)
        (wv * x).sum().backward()
        return b.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    xf = torch.zeros_like(b0)
    fwd = mg.pressure_solve(h, b0, xf, tol=args.tol)
    adj = mg.pressure_solve_adjoint(h, wv, torch.zeros_like(b0), tol=args.tol)
    line = {
        "metric": f"ms per forward + backward pressure solve (autograd) at C{cfg.n}L{cfg.nlev}",
        "value": round(ms, 4), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": f"{workload_name(cfg, args.precision)}; loss <w, x>, dL/db by the adjoint solve",
                   "forward_iters": fwd.iters, "adjoint_iters": adj.iters},
        "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.destroy()


def run_mixed_adjoint(args, cfg, inp, mg, torch, world, rank):
    """The differentiable mixed solve: forward (u, p) = A^-1 rhs and backward dL/drhs = A^-T
    dL/d(u, p) through the torch autograd wrapper, L = <w_u, u> + <w_p, p> (C48L30 by default)."""
    h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=True)
    ru0 = torch.from_numpy(inp["rhs_u"]).cuda()
    rp0 = torch.from_numpy(inp["rhs_p"]).cuda()
    wu = torch.from_numpy(syn.normal(cfg.seed, 98, ru0.numel())).cuda()
    wp = torch.from_numpy(syn.normal(cfg.seed, 99, rp0.numel())).cuda()

    def step():
        ru = ru0.clone().requires_grad_(True)
        rp = rp0.clone().requires_grad_(True)
        u, p = mg.solve_mixed(h, ru, rp, tol=args.tol)
        ((wu * u).sum() + (wp * p).sum()).backward()
        return ru.grad, rp.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fwd = mg.mixed_solve(h, ru0, rp0, torch.zeros_like(ru0), torch.zeros_like(rp0), tol=args.tol)
    adj = mg.mixed_solve_adjoint(h, wu, wp, torch.zeros_like(ru0), torch.zeros_like(rp0), tol=args.tol)
    line = {
        "metric": f"ms per forward + backward mixed (u, p) solve (autograd) at {cfg.name.upper()}",
        "value": round(ms, 4), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": f"{cfg.name} mixed system (eps = {cfg.eps}"
                               + (", consistent velocity mass" if cfg.consistent_mass else "")
                               + (f", rotation {cfg.rotation:g}/s" if cfg.rotation else "")
                               + f"), {cfg.levels}-level {args.precision} V-cycle; loss <w, (u, p)>, dL/drhs "
                                 "by the adjoint solve",
                   "forward_iters": fwd.iters, "adjoint_iters": adj.iters},
        "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.destroy()


ENSEMBLE = [(n, nlev) for n in (32, 40, 48, 64, 80, 96, 112, 128) for nlev in (30, 50, 70)]


def run_ensemble(args, mg, torch, world, rank):
    """24 independent pressure solves (C32-C128 x 30 / 50 / 70 levels, 4-level FP32 V-cycle,
    GCR(5) FP64), solved one after the other through pressure_solve, together through
    ensemble_pressure_solve (interleaved iterations, one stream per member) and as one graph
    launch through mg_ensemble (the value)."""
    hs, bs, xs = [], [], []
    for i, (n, nlev) in enumerate(ENSEMBLE):
        cfg = syn.small_config(n, nlev, levels=4, seed=syn.BASE_SEED + 200 + i)
        inp = syn.make_inputs(cfg, mixed=False)
        hs.append(mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=False))
        bs.append(torch.from_numpy(inp["rhs"]).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    cells = sum(int(b.numel()) for b in bs)
    for _ in range(args.warmup):
        for h, b, x in zip(hs, bs, xs):
            mg.pressure_solve(h, b, x, tol=args.tol)
        mg.ensemble_pressure_solve(hs, bs, xs, tol=args.tol)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the ensemble with the built-in launch shapes, then every member autotuned (untimed)
    e0.record()
    for _ in range(args.steps):
        mg.ensemble_pressure_solve(hs, bs, xs, tol=args.tol)
    e1.record()
    torch.cuda.synchronize()
    untuned_ms = e0.elapsed_time(e1) / args.steps
    tuned = [mg.mg_autotune(h) for h in hs]
    for h, b, x in zip(hs, bs, xs):
        mg.pressure_solve(h, b, x, tol=args.tol)   # recapture the per-iteration graphs
    mg.ensemble_pressure_solve(hs, bs, xs, tol=args.tol)
    torch.cuda.synchronize()
    # the whole ensemble as one CUDA graph (created after tuning: it records the launch shapes)
    ens = mg.Ensemble(hs, bs, xs, tol=args.tol)
    for _ in range(args.warmup):
        ens.solve()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        e0.record()
        for _ in range(args.steps):
            for h, b, x in zip(hs, bs, xs):
                mg.pressure_solve(h, b, x, tol=args.tol)
        e1.record()
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1) / args.steps
        lat_i = []
        e0.record()
        for _ in range(args.steps):
            infos = mg.ensemble_pressure_solve(hs, bs, xs, tol=args.tol)
            lat_i += [i.ms for i in infos]
            assert all(i.converged for i in infos), infos
        e1.record()
        torch.cuda.synchronize()
        inter_ms = e0.elapsed_time(e1) / args.steps
        lat = []
        e0.record()
        for _ in range(args.steps):
            infos = ens.solve()
            lat += [i.ms for i in infos]
            assert all(i.converged for i in infos), infos
        e1.record()
        torch.cuda.synchronize()
        ens_ms = e0.elapsed_time(e1) / args.steps
    ens.destroy()
    lat = np.sort(np.array(lat))
    lat_i = np.sort(np.array(lat_i))
    line = {
        "metric": "members per second, 24-member pressure-solve ensemble (C32-C128 x 30/50/70 levels)",
        "value": round(len(hs) / (ens_ms * 1e-3), 2), "unit": "members/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ens_ms, 3), "higher_is_better": True,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": f"24 members, n in (32..128), nlev in (30, 50, 70), 4-level {args.precision} "
                               f"V-cycle, GCR(5), tol {args.tol:g}; one graph launch per ensemble solve "
                               "(mg_ensemble, device-side convergence decisions)",
                   "cells": cells, "members": len(hs), "gpu_launches_per_step": 1},
        "sequential": {"members_per_s": round(len(hs) / (seq_ms * 1e-3), 2), "ms": round(seq_ms, 3)},
        "interleaved_streams": {"members_per_s": round(len(hs) / (inter_ms * 1e-3), 2), "ms": round(inter_ms, 3),
                                "member_latency_ms": {"p50": round(float(np.percentile(lat_i, 50)), 3),
                                                      "p99": round(float(np.percentile(lat_i, 99)), 3)}},
        "speedup_vs_sequential": round(seq_ms / ens_ms, 3),
        "autotune": {"note": "value and sequential use the launch shapes mg_autotune chose per member and level",
                     "untuned_ensemble_ms": round(untuned_ms, 3),
                     "speedup_vs_untuned": round(untuned_ms / ens_ms, 3),
                     "finest_level_choices": sorted({tuple(t[0]) for t in tuned})},
        "member_latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                              "p99": round(float(np.percentile(lat, 99)), 3), "max": round(float(lat[-1]), 3)},
        "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for h in hs:
        h.destroy()


# Table 1 of the paper: (name, levels of the handle, pressure solver kind, eps_H, omega, sweeps)
SOLVER_TABLE = [
    ("line relaxation", 4, "jacobi", 0.0, 0.8, 10),
    ("Krylov(1e-2)", 4, "bicgstab_jacobi", 1e-2, 1.0, 1),
    ("Krylov(1e-3)", 4, "bicgstab_jacobi", 1e-3, 1.0, 1),
    ("Krylov(1e-6)", 4, "bicgstab_jacobi", 1e-6, 1.0, 1),
    ("MG(1)", 1, "mg", 0.0, 0.8, 0),
    ("MG(2)", 2, "mg", 0.0, 0.8, 0),
    ("MG(3)", 3, "mg", 0.0, 0.8, 0),
    ("MG(4)", 4, "mg", 0.0, 0.8, 0),
    ("Kr-MG(1e-2,4)", 4, "bicgstab_mg", 1e-2, 0.8, 0),
    ("Kr-MG(1e-3,4)", 4, "bicgstab_mg", 1e-3, 0.8, 0),
    ("Kr-MG(1e-6,4)", 4, "bicgstab_mg", 1e-6, 0.8, 0),
]


def run_solver_table(args, cfg, inp, mg, torch, world, rank):
    """The paper's pressure-solver comparison (Table 1 configurations, Table 2 quantities) on the
    mixed workload: per configuration the outer GCR iterations per mixed solve, the BiCGStab
    iterations per pressure solve, ms per mixed solve and ms per pressure solve alone."""
    ru = torch.from_numpy(inp["rhs_u"]).cuda()
    rp = torch.from_numpy(inp["rhs_p"]).cuda()
    rows = []
    with Clocks(0) as clk:
        for name, levels, kind, eps, omega, sweeps in SOLVER_TABLE:
            h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=True, levels=levels)
            mg.mg_set_pressure_solver(h, kind, eps=eps, omega=omega, sweeps=sweeps, max_iter=500)
            u, p = torch.zeros_like(ru), torch.zeros_like(rp)
            for _ in range(args.warmup):
                mg.mixed_solve(h, ru, rp, u, p, tol=args.tol)
            mg.mg_inner_stats(h)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            its = []
            e0.record()
            for _ in range(args.steps):
                info = mg.mixed_solve(h, ru, rp, u, p, tol=args.tol)
                assert info.converged, (name, info)
                its.append(info.iters)
            e1.record()
            torch.cuda.synchronize()
            ms_mixed = e0.elapsed_time(e1) / args.steps
            nsolve, inner = mg.mg_inner_stats(h)
            x = torch.zeros_like(rp)
            e0.record()
            for _ in range(args.steps):
                mg.helmholtz_solve(h, rp, x)
            e1.record()
            torch.cuda.synchronize()
            ms_press = e0.elapsed_time(e1) / args.steps
            rows.append({"pressure_solver": name, "outer_iters": statistics.mean(its),
                         "inner_iters": round(inner / nsolve, 2) if nsolve else None,
                         "ms_mixed": round(ms_mixed, 3), "ms_pressure": round(ms_press, 4)})
            h.destroy()
    cfl = cfg.cs * cfg.dt / (0.5 * np.pi * cfg.radius / cfg.n)
    line = {
        "metric": f"pressure-solver comparison (Table 1 configurations) on the {cfg.name.upper()} mixed system",
        "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": f"C{cfg.n}L{cfg.nlev} mixed system, eps = {cfg.eps}, dt = {cfg.dt:g} s "
                               f"(CFL_h = {cfl:.1f}), outer GCR(5) to {args.tol:g}, {args.precision} V-cycles "
                               "and block-Jacobi sweeps"},
        "table": rows, "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_mixed(args, cfg, inp, mg, torch, world, rank):
    """The mixed (u, p) solve: GCR(5) on the reduced mixed operator, right-preconditioned by the
    Schur-complement step with one V-cycle (Sec. 3.4, 4.1), from zero to 1e-8."""
    h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=True)
    ru = torch.from_numpy(inp["rhs_u"]).cuda()
    rp = torch.from_numpy(inp["rhs_p"]).cuda()
    u, p = torch.zeros_like(ru), torch.zeros_like(rp)
    for _ in range(args.warmup):
        info = mg.mixed_solve(h, ru, rp, u, p, tol=args.tol)
        assert info.converged, info
    # untimed: every launch of a few solves
    n_prof = 3
    mg.mg_profile_start(h, 1 << 16)
    for _ in range(n_prof):
        mg.mixed_solve(h, ru, rp, u, p, tol=args.tol)
    recs = mg.mg_profile_stop(h)
    by = {}
    for r in recs:
        a = by.setdefault((r["kind"], r["level"]), [0, 0.0, 0.0])
        a[0] += 1
        a[1] += r["ms"]
        a[2] += r["bytes"]
    total = sum(v[1] for v in by.values())
    (kind, lev), (cnt, ms, byt) = max(by.items(), key=lambda kv: kv[1][1])
    peak, peak_src = _peaks()
    # timed region
    torch.cuda.synchronize()
    iters = []
    with Clocks(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            info = mg.mixed_solve(h, ru, rp, u, p, tol=args.tol)
            iters.append(info.iters)
        e1.record()
        torch.cuda.synchronize()
    ms_solve = e0.elapsed_time(e1) / args.steps
    line = {
        "metric": f"ms per mixed (u, p) solve to {args.tol:g} rel. residual at {cfg.name.upper()}",
        "value": round(ms_solve, 4), "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": f"{cfg.name} mixed system (eps = {cfg.eps}"
                               + (", consistent velocity mass" if cfg.consistent_mass else "")
                               + (f", rotation {cfg.rotation:g}/s" if cfg.rotation else "")
                               + f"), GCR(5) + Schur-complement {cfg.levels}-level {args.precision} V-cycle",
                   "n": cfg.n, "nlev": cfg.nlev,
                   "unknowns_u": int(ru.numel()), "unknowns_p": int(rp.numel()),
                   "iters_per_solve": statistics.mean(iters)},
        "roofline": {"bound": "hbm", "kernel": f"{kind}@L{lev}", "achieved": round(byt / (ms * 1e-3) / 1e9, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(byt / (ms * 1e-3) / 1e9 / peak, 4),
                     "peak_source": peak_src, "timing": f"CUDA events around every launch of {n_prof} untimed solves"},
        "kernels": {f"{k[0]}@L{k[1]}": {"launches": v[0] // n_prof, "ms": round(v[1] / n_prof, 4),
                                        "share": round(v[1] / total, 4),
                                        "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1)}
                    for k, v in sorted(by.items(), key=lambda kv: -kv[1][1])},
        "clocks": clk.result,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.destroy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c192")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32_p64", "fp32_bf16"])
    ap.add_argument("--dt", type=float, default=None,
                    help="time step in s (default: the workload's, 600 s; 1200 s gives CFL_h ~ 7.9 at C192, "
                         "the paper's regime for the robustness sweep)")
    ap.add_argument("--levels", type=int, default=None, help="multigrid levels (default: the workload's)")
    ap.add_argument("--system", default="pressure", choices=["pressure", "mixed", "ensemble", "adjoint",
                                                             "mixed_adjoint", "solvers"],
                    help="mixed: the (u, p) solve (GCR + Schur-complement multigrid) on the C48L30 "
                         "mixed workload instead of the headline pressure solve")
    ap.add_argument("--tol", type=float, default=SOLVE_TOL)
    ap.add_argument("--consistent-mass", action="store_true",
                    help="mixed system: consistent RT0 velocity mass instead of the lumped one")
    ap.add_argument("--rotation", type=float, default=0.0,
                    help="mixed system: planet angular velocity [1/s] of the implicit Coriolis term")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare-precisions", dest="compare_precisions", action="store_false",
                    help="skip timing the FP64-pivot and plain FP64 V-cycle solves beside the FP32 one")
    ap.add_argument("--profile-solve", action="store_true",
                    help="untimed: one pressure solve limited to --iters GCR iterations (for ncu captures)")
    ap.add_argument("--iters", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_init()
    if args.system in ("mixed", "mixed_adjoint", "solvers") and args.workload == "c192":
        args.workload = "c48"
    if args.system == "adjoint" and args.workload == "c192":
        args.workload = "c96"
    if args.impl == "reference" and args.system in ("ensemble", "adjoint", "mixed_adjoint", "solvers"):
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the pressure solve "
                                                                  "only (the headline metric)"}))
        return
    cfg = syn.config(args.workload)
    if args.dt is not None or args.levels is not None:
        import dataclasses
        cfg = dataclasses.replace(cfg, dt=args.dt or cfg.dt, levels=args.levels or cfg.levels)
    if args.consistent_mass or args.rotation:
        import dataclasses
        cfg = dataclasses.replace(cfg, consistent_mass=args.consistent_mass, rotation=args.rotation)
    inp = syn.make_inputs(cfg, mixed=args.system in ("mixed", "mixed_adjoint", "solvers"))
    if args.impl == "reference" and args.system == "mixed":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the pressure solve "
                                                                  "only (the headline metric)"}))
        return
    if args.impl == "reference":
        return run_reference(args, cfg, inp, world, rank)

    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2002_00756_gb300.build import build
    if rank == 0:
        build()
    if pg:
        pg.barrier()
    import paper_2002_00756_gb300 as mg

    if args.system == "mixed":
        return run_mixed(args, cfg, inp, mg, torch, world, rank)
    if args.system == "solvers":
        return run_solver_table(args, cfg, inp, mg, torch, world, rank)
    if args.system == "ensemble":
        return run_ensemble(args, mg, torch, world, rank)
    if args.system == "adjoint":
        return run_adjoint(args, cfg, inp, mg, torch, world, rank)
    if args.system == "mixed_adjoint":
        return run_mixed_adjoint(args, cfg, inp, mg, torch, world, rank)

    if args.profile_solve:
        h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=False, max_iter=args.iters)
        b = torch.from_numpy(inp["rhs"]).cuda()
        info = mg.pressure_solve(h, b, torch.zeros_like(b), tol=args.tol)
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve": args.workload, "iters": info.iters, "rel_res": info.rel_res}))
        h.destroy()
        return
    h = mg.mg_setup_config(cfg, inp, precision=args.precision, mixed=False)
    stream = torch.cuda.current_stream()
    b = torch.from_numpy(inp["rhs"]).cuda()
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        info = mg.pressure_solve(h, b, x, tol=args.tol)
        assert info.converged, info
    torch.cuda.synchronize()

    # ---- untimed: every launch of a few solves, for the kernel breakdown ----
    n_prof = 3
    mg.mg_profile_start(h, 1 << 16)
    for _ in range(n_prof):
        mg.pressure_solve(h, b, x, tol=args.tol)
    all_recs = mg.mg_profile_stop(h)
    by, byv = {}, {}
    for r in all_recs:
        for key, dct in (((r["kind"], r["level"]), by), ((r["kind"], r["level"], r["variant"]), byv)):
            a = dct.setdefault(key, [0, 0.0, 0.0])
            a[0] += 1
            a[1] += r["ms"]
            a[2] += r["bytes"]
    # the dominant kernel: the single kernel (kind, level, variant) with the most time
    (kind, lev, var) = max(byv.items(), key=lambda kv: kv[1][1])[0]

    # ---- timed region: K solves, inputs resident in HBM ----
    iters = []
    with Clocks(local) as clk:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            info = mg.pressure_solve(h, b, x, tol=args.tol)
            iters.append(info.iters)
        e1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    ms_total = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
    ms_per_solve = job_ms_per_unit(ms_total, args.steps, world)

    # ---- e2e: host buffers through the public API ----
    bh = torch.from_numpy(inp["rhs"]).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    bd = torch.empty_like(b)
    xd = torch.empty_like(b)
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bd.copy_(bh, non_blocking=True)
        mg.pressure_solve(h, bd, xd, tol=args.tol)
        xh.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = job_ms_per_unit(max_over_ranks((time.perf_counter() - t0) * 1e3, pg, "cuda"), e2e_steps, world)

    # ---- the same solve with the finest level eliminated in FP64 (MG_FP32_P64) and with the
    # plain FP64 V-cycle, a few solves each, timed the same way ----
    compare = {}
    if args.precision == "fp32" and args.compare_precisions:
        for prec in ("fp32_p64", "fp64"):
            hc = mg.mg_setup_config(cfg, inp, precision=prec)
            xc = torch.zeros_like(b)
            for _ in range(2):
                mg.pressure_solve(hc, b, xc, tol=args.tol)
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nc = 3
            c0.record(stream)
            for _ in range(nc):
                ic = mg.pressure_solve(hc, b, xc, tol=args.tol)
            c1.record(stream)
            torch.cuda.synchronize()
            compare[prec] = {"ms_per_solve": round(c0.elapsed_time(c1) / nc, 3), "iters": ic.iters,
                             "rel_res": float(f"{ic.rel_res:.3e}")}
            hc.destroy()

    # ---- roofline of the dominant kernel: K more solves, timed the same way, with CUDA
    # events around every launch of the dominant kernel's kind and level (the solves then
    # run as plain launches instead of the cached per-iteration graphs) ----
    mg.mg_profile_start(h, 1 << 16, kind=kind, level=lev)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        mg.pressure_solve(h, b, x, tol=args.tol)
    recs = mg.mg_profile_stop(h)
    peak, peak_src = _peaks()
    sel = [r for r in recs if (r["kind"], r["level"], r["variant"]) == (kind, lev, var)]
    cnt, ms, byt = len(sel), sum(r["ms"] for r in sel), sum(r["bytes"] for r in sel)
    kname = f"{kind}@L{lev}" + (f"/{SWEEP_VARIANTS[var]}" if kind == "sweep" else
                                (f"/J{var}" if kind == "apply" else ""))
    achieved = byt / (ms * 1e-3) / 1e9
    traffic = profiled_traffic(kname, cfg.name, args.precision)
    roof = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4)}
    if kind == "apply":
        # the fused FP64 apply issues 7 FP64 instructions per cell for H z in diagonal form
        # (1 multiply, 6 fused multiply-adds) plus J + 2 for the GCR sums; the bound is the
        # FP64 issue rate: 152 SMs x 2 per clock x 2.07 GHz
        fp64_peak = 152 * 2 * 2.07                      # G FP64 instructions / s
        inst = (7 + var + 2) * cfg.ncell * cnt
        ach = inst / (ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": kname, "achieved": round(ach, 1), "peak": round(fp64_peak, 1),
                "unit": "G FP64 inst/s", "frac": round(ach / fp64_peak, 4), "hbm_GBps": round(achieved, 1),
                "hbm_frac": round(achieved / peak, 4)}
    vc_kinds = ("sweep", "restrict", "prolong", "convert")
    vc_ms = sum(v[1] for k, v in by.items() if k[0] in vc_kinds)
    vc_bytes = sum(v[2] for k, v in by.items() if k[0] in vc_kinds)
    total_kernel_ms = sum(v[1] for v in by.values())
    breakdown = {f"{k[0]}@L{k[1]}": {"launches": v[0] // n_prof, "ms": round(v[1] / n_prof, 4),
                                     "share": round(v[1] / total_kernel_ms, 4),
                                     "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1)}
                 for k, v in sorted(by.items(), key=lambda kv: -kv[1][1])}

    line = {
        "metric": METRIC, "value": round(ms_per_solve, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": {"workload": workload_name(cfg, args.precision) if args.tol == SOLVE_TOL else
                   workload_name(cfg, args.precision).split(", stopped")[0] + f", tol {args.tol:g}",
                   "n": cfg.n, "nlev": cfg.nlev, "unknowns": cfg.ncell, "levels": cfg.levels, "dt_s": cfg.dt,
                   "vcycle_precision": args.precision, "tol": args.tol, "gcr_restart": cfg.gcr_restart,
                   "iters_per_solve": statistics.mean(iters), "replicas": world,
                   "l2": "working set (~3 GB) larger than L2; no flush"},
        "e2e": {"value": round(e2e_ms, 4), "unit": UNIT, "h2d_bytes_per_step": int(b.numel() * 8),
                "d2h_bytes_per_step": int(b.numel() * 8)},
        "roofline": {**roof,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per launch (ncu)", "algorithmic_bytes_per_launch": round(byt / cnt),
                     "launch_us": round(ms / cnt * 1e3, 2), "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "timing": f"CUDA events around each of the {cnt} launches of this kernel in {args.steps} "
                               f"further solves (launched directly, not from the per-iteration graphs)",
                     "vcycle_GBps": round(vc_bytes / (vc_ms * 1e-3) / 1e9, 1),
                     "vcycle_frac": round(vc_bytes / (vc_ms * 1e-3) / 1e9 / peak, 4)},
        "gpu_launches": len(all_recs) // n_prof * args.steps,
        **({"compare_precisions": {"note": "the same solve, 3 timed after 2 untimed; fp32_p64: FP32 V-cycle "
                                           "with the finest level's column elimination in FP64; fp64: the "
                                           "plain FP64 V-cycle", **compare}} if compare else {}),
        "kernels": {"note": f"per solve, from {n_prof} untimed solves with every launch event-timed", **breakdown},
        "clocks": clk.result,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if cfg.name == "c192" and cfg.dt == 600.0 and cfg.levels == 4:
            full, cores = cpu_baseline_full(args.tol)
            c = full["c192"]
            line["cpu_baseline"] = {
                "value": c["ms_per_solve_1core"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "iters": c["iters"],
                "sample": f"one complete oracle solve of the same C192L70 problem to {args.tol:g} (numpy FP64, "
                          f"its own {c['iters']} GCR iterations, set-up of {c['setup_s']} s not counted), one core; "
                          f"host has {cores} cores (nproc): C12L30, C48L30 and C96L70 pressure solves on 1 core and on all "
                          "cores at once (one process per core) in 'workloads'",
                "workloads": full, "host_cores": cores}
        else:
            sec_it, hist = cpu_oracle_iteration_time(cfg, inp, iters=1)
            n_it = statistics.mean(iters)
            line["cpu_baseline"] = {
                "value": round(sec_it * n_it * 1e3, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"one numpy FP64 GCR iteration of the same solve ({sec_it:.1f} s) x "
                          f"{n_it:.1f} iterations per solve (the GPU solve's count)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.destroy()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
