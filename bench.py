#!/usr/bin/env python
"""Benchmark of the EREM / real-Leja phi_1 path on one GB300.

Workload (default): the 256^3 layered reservoir with 8 x-aligned
high-permeability channels (contrast 1e4), Peclet 1e3, dt = 1/32, Leja
tolerance 1e-6; one "step" is one EREM step (eq. EERM): G(T^n), the fused
Leja terms with their device-side stopping test, and the update.  The Darcy
field is frozen (one pressure solve in set-up), so the Jacobian and its
Gershgorin interval are assembled once, outside the timed region.

Headline: FP32-bulk Mcell-steps/s (cells x steps / device time).  Also
reported: the plain FP64 form on the same steps (ratio and relative L2
difference of the two results), the end-to-end rate through the C ABI with
host buffers, the roofline of the Leja term kernel (algorithmic bytes per
cell-term over its CUDA-event time against the measured HBM copy bandwidth),
SM clocks sampled during the timed region, and the CPU oracle timed on a
bounded slab of the same workload.

With --impl reference the CPU oracle itself is timed (each step one oracle
EREM step on a 256 x 256 x 16 slab of the workload, all its channels kept).
Under torchrun every rank runs an independent replica on its own GPU (the
single-grid path is not sharded): value = all ranks' cell-steps / max time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EREM Mcell-steps/s at 256³ FP32-bulk vs FP64 at ≤1e-5 rel err; HBM GB/s vs peak"
UNIT = "Mcell-steps/s"
# algorithmic bytes per cell of one Leja term (3D): 7 coefficients, q read,
# q written, P read and written (FP64)
BYTES_PER_CELL_TERM = {"fp32_bulk": 7 * 4 + 4 + 4 + 16, "fp64": 7 * 8 + 8 + 8 + 16}
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="grid cells per direction")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-krylov", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--slab", type=int, default=16, help="z planes of the oracle's sample")
    ap.add_argument("--workload", choices=["channels3d", "coupled2d", "ensemble", "adjoint"],
                    default="channels3d",
                    help="channels3d: the 256^3 headline; coupled2d: 1024^2 sequential "
                         "pressure/temperature with T-dependent fluid laws; ensemble: 512 "
                         "independent 2D members of 64^2..512^2 cells in one batched run")
    ap.add_argument("--members", type=int, default=512, help="ensemble members")
    ap.add_argument("--arms", default="all",
                    help="coupled2d: comma-separated subset of erem_fp32_bulk, erem_fp64, ros2_fp64, "
                         "ros3p_fp64, erem_strang_fp32_bulk, erem_from_last_fp32_bulk (the line "
                         "needs erem_fp32_bulk)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate(ms_local: float, cells: int, steps: int, world: int, device=None):
    """Whole-job rate of `world` replicas that each ran `steps` steps over
    `cells` cells: the slowest rank's time sets the job time.  Returns
    (max ms over ranks, Mcell-steps/s of all ranks)."""
    ms = max_over_ranks(ms_local, world, device)
    return ms, world * cells * steps / (ms / 1e3) / 1e6


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_sources_sha():
    """Hash of the source the Leja term kernel is built from: the shared
    device helpers and the k_leja_term definition itself."""
    csrc = os.path.join(ROOT, "paper_1209_5553_gb300", "csrc")
    kern = open(os.path.join(csrc, "kernels.cu")).read()
    start = kern.index("k_leja_term(const Tq* __restrict__ qi")
    end = kern.index("\n}\n", start)
    h = hashlib.sha256()
    h.update(open(os.path.join(csrc, "device_common.cuh"), "rb").read())
    h.update(kern[start:end].encode())
    return h.hexdigest()[:16]


def recorded_traffic(precision: str, n_cells: int):
    """Bytes per Leja-term launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"k_leja_term_{precision}_channels3d_{round(n_cells ** (1 / 3))}.md")
    try:
        sha = kernel_sources_sha()
        vals = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(": ", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel sources sha256[:16]") != sha:
            return None
        return float(vals["dram bytes per cell-term"]) * n_cells
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------
def make_workload(n):
    import workloads as W

    return W.channels3d(n)


def linear_head(n, nx, head_left, head_right):
    """Pressure initial guess: the head interpolated linearly in x."""
    x = (np.arange(nx) + 0.5) / nx
    ramp = head_left + (head_right - head_left) * x
    return np.broadcast_to(ramp, (n // nx, nx)).reshape(-1).copy()


def gpu_context(E, torch, wl, precision, dev):
    """Context with the workload's state set: GPU pressure solve, velocity
    scaling (largest face speed 1), heat capacity for Pe = 1e3."""
    n = wl.n
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    ctx = E.Context(3, wl.nx, wl.ny, wl.nz, physics=E.Physics(1.0, 1.0, wl.head_drop, 0.0,
                                                             wl.T_inflow, 0),
                    precision=precision)
    lnk = t(wl.lnk)
    p = t(linear_head(n, wl.nx, wl.head_drop, 0.0))
    st = ctx.pressure_solve(lnk, None, p, tol=1e-10, maxit=200000)
    import workloads as W

    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), 1.0)
    head = wl.head_drop / st.vmax
    ctx.set_physics(E.Physics(rc, rc, head, 0.0, wl.T_inflow, 0))
    p = t(linear_head(n, wl.nx, head, 0.0))
    st2 = ctx.pressure_solve(lnk, None, p, tol=1e-10, maxit=200000)
    T = t(wl.T0)
    ctx.set_state(T, p, lnk, t(wl.phi), t(wl.lam), wl.dt)
    return ctx, T, {"pressure_iters": [st.lin_iters, st2.lin_iters], "vmax_unscaled": st.vmax,
                    "rhoc": rc, "head_left": head}


def run_gpu(E, torch, wl, precision, steps, warmup, dev, world, sample_clocks=False, points="exact"):
    ctx, T, info = gpu_context(E, torch, wl, precision, dev)
    ctx.set_leja_points(points)
    opts = E.leja_opts(tol=wl.tol, time_terms=True)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.erem_step(T, wl.dt, opts=opts)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(dev.index if dev.index is not None else 0) if sample_clocks else None
    if sampler:
        sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    degrees, t_terms, n_terms, n_leja, launches = [], 0.0, 0, 0, 0
    t0.record(stream)
    for _ in range(steps):
        st = ctx.erem_step(T, wl.dt, opts=opts)
        degrees.append(st.schedule)
        t_terms += st.t_terms_ms
        n_terms += st.n_terms_timed
        n_leja += st.n_launches_timed
        launches += st.launches
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    barrier(world)
    out = {"ms": ms, "degrees": degrees, "t_terms_ms": t_terms, "n_terms": n_terms,
           "n_leja": n_leja, "launches": launches, "T": T.cpu().numpy(), "clocks": clocks, "info": info,
           "alpha": st.alpha, "beta": st.beta}
    ctx.close()
    return out


def run_forced(E, torch, wl, steps, warmup, dev):
    """The same workload with a time-dependent inflow temperature
    T_in(t) = 60 + 20 sin(2 pi t) (eq. nEERMg: phi_1 and phi_2 per step),
    FP32-bulk."""
    import math

    ctx, T, _ = gpu_context(E, torch, wl, "fp32_bulk", dev)
    opts = E.leja_opts(tol=wl.tol)
    tin = lambda t: 60.0 + 20.0 * math.sin(2 * math.pi * t)
    rate = lambda t: 40.0 * math.pi * math.cos(2 * math.pi * t)
    k = 0
    for _ in range(warmup):
        ctx.erem_step_forced(T, wl.dt, tin(k * wl.dt), rate(k * wl.dt), opts=opts)
        k += 1
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    terms1, terms2 = [], []
    e0.record(stream)
    for _ in range(steps):
        st = ctx.erem_step_forced(T, wl.dt, tin(k * wl.dt), rate(k * wl.dt), opts=opts)
        terms1.append(st.degree_total - st.degree_phi2)
        terms2.append(st.degree_phi2)
        k += 1
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"ms": e0.elapsed_time(e1), "phi1_terms_per_step": float(np.mean(terms1)),
           "phi2_terms_per_step": float(np.mean(terms2))}
    ctx.close()
    return out


def run_krylov(E, torch, wl, steps, warmup, dev):
    """The same steps with phi_1 by Krylov substeps (FP64, §4.1)."""
    ctx, T, _ = gpu_context(E, torch, wl, "fp64", dev)
    opts = E.krylov_opts(tol=wl.tol)
    for _ in range(warmup):
        ctx.erem_step_krylov(T, wl.dt, opts=opts)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    subs, rej, launches = [], 0, 0
    e0.record(stream)
    for _ in range(steps):
        st = ctx.erem_step_krylov(T, wl.dt, opts=opts)
        subs.append(st.substeps)
        rej += st.rejections
        launches += st.launches
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"ms": e0.elapsed_time(e1), "substeps_per_step": subs, "rejections": rej,
           "launches": launches, "T": T.cpu().numpy()}
    ctx.close()
    return out


def run_e2e(E, torch, wl, steps, warmup, dev):
    """Same steps through the C ABI with a pinned host T: the library copies
    T to the device and the result back inside every call."""
    ctx, Td, _ = gpu_context(E, torch, wl, "fp32_bulk", dev)
    T = torch.empty(wl.n, dtype=torch.float64).pin_memory()
    T.copy_(Td.cpu())
    opts = E.leja_opts(tol=wl.tol)
    for _ in range(warmup):
        ctx.erem_step(T, wl.dt, opts=opts)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        ctx.erem_step(T, wl.dt, opts=opts)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t
    ctx.close()
    return sec


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample: a 16-plane z slab holding channels
# ---------------------------------------------------------------------------
def oracle_sample(wl, nz_s):
    from oracle import fv, timestep as ts
    import workloads as W

    n = wl.nx
    lnk = wl.lnk.reshape(wl.nz, wl.ny, wl.nx)
    chan = np.isclose(lnk, np.log(1e4)).sum(axis=(1, 2))
    starts = list(range(0, wl.nz - nz_s + 1, nz_s))
    z0 = max(starts, key=lambda z: chan[z:z + nz_s].sum())
    sl = slice(z0, z0 + nz_s)
    f = lambda a: np.ascontiguousarray(a.reshape(wl.nz, wl.ny, wl.nx)[sl]).reshape(-1)
    g = fv.Grid(3, n, wl.ny, nz_s, 1.0, 1.0, nz_s / wl.nz)
    base = fv.Physics(head_left=wl.head_drop, head_right=0.0, T_inflow=wl.T_inflow)
    slnk = f(wl.lnk)
    p, _, _ = ts.pressure_solve_cg(g, base, slnk, tol=1e-10)
    vx, vy, vz = fv.darcy_fluxes(g, base, slnk, p)
    a = g.face_area
    vmax = max(np.abs(vx).max() / a[0], np.abs(vy).max() / a[1], np.abs(vz).max() / a[2])
    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), 1.0)
    phys = fv.Physics(rc, rc, wl.head_drop / vmax, 0.0, wl.T_inflow, 0)
    prob = ts.heat_problem(g, phys, slnk, f(wl.phi), f(wl.lam), p / vmax)
    return prob, f(wl.T0), g.n, f"z-slab {n}x{wl.ny}x{nz_s} (planes {z0}..{z0 + nz_s - 1}) of the {wl.nx}^3 workload"


def time_oracle(wl, nz_s, steps, warmup=0):
    from oracle import timestep as ts
    from oracle.leja import LejaOptions

    prob, T, ncell, desc = oracle_sample(wl, nz_s)
    opts = LejaOptions(tol_a=wl.tol, tol_r=wl.tol)
    for _ in range(warmup):
        T, _ = ts.erem_step(prob, T, wl.dt, opts)
    t = time.perf_counter()
    for _ in range(steps):
        T, _ = ts.erem_step(prob, T, wl.dt, opts)
    sec = time.perf_counter() - t
    return ncell * steps / sec / 1e6, sec, ncell, desc


def oracle_threads():
    # numpy elementwise work and scipy's sparse products run on one thread
    return 1


# ---------------------------------------------------------------------------
def main_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    wl = make_workload(args.n)
    value, sec, ncell, desc = time_oracle(wl, args.slab, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"channels3d_{args.n}", "sample": desc, "dt": wl.dt, "tol": wl.tol},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"{args.steps} oracle EREM steps on the {desc}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(args):
    rank, world, local = dist_info()
    import torch

    import paper_1209_5553_gb300 as E

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init(world, "nccl")
    wl = make_workload(args.n)
    N = wl.n
    K, Wu = args.steps, args.warmup

    r32 = run_gpu(E, torch, wl, "fp32_bulk", K, Wu, dev, world, sample_clocks=(rank == 0))
    ms, value = aggregate(r32["ms"], N, K, world, dev)
    peak, peak_kind = measured_peaks()
    b32 = BYTES_PER_CELL_TERM["fp32_bulk"]
    # one Leja term must move the coefficients once, q in and out, and P in
    # and out: 52 B per cell
    sec_leja = r32["t_terms_ms"] / 1e3
    achieved = b32 * N * r32["n_leja"] / sec_leja / 1e9 if r32["n_leja"] else None
    effective = b32 * N * r32["n_terms"] / sec_leja / 1e9 if r32["n_terms"] else None
    traffic = recorded_traffic("fp32_bulk", N)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wu,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"channels3d_{args.n}", "grid": [args.n] * 3, "cells": N,
                   "dt": wl.dt, "tol": wl.tol, "peclet": wl.peclet,
                   "precision": "fp32_bulk: FP32 stencil and Leja vectors; FP64 divided differences, "
                                "interval, running sum and error estimate",
                   "l2": "inputs larger than L2 (coefficients + vectors ~1.3 GB per term)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": r32["clocks"],
        "gpu_launches": r32["launches"],
        "leja": {"degrees_per_step": [s[1:] if s[0] == 1 else s for s in r32["degrees"]],
                 "terms_timed": r32["n_terms"], "alpha": r32["alpha"], "beta": r32["beta"]},
        "roofline": {"kernel": "k_leja_term<float,4,3>",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_cell_per_launch": b32,
                     "launch_ms_avg": r32["t_terms_ms"] / max(r32["n_leja"], 1),
                     "terms_per_launch": r32["n_terms"] / max(r32["n_leja"], 1),
                     "effective_gbs_per_term": effective,
                     "term_ms_avg": r32["t_terms_ms"] / max(r32["n_terms"], 1)},
        "setup": r32["info"],
    }
    if not args.no_fp64:
        r64 = run_gpu(E, torch, wl, "fp64", K, Wu, dev, world)
        ms64, value64 = aggregate(r64["ms"], N, K, world, dev)
        b64 = BYTES_PER_CELL_TERM["fp64"]
        ach64 = b64 * N * r64["n_leja"] / (r64["t_terms_ms"] / 1e3) / 1e9 if r64["n_leja"] else None
        rel = float(np.linalg.norm(r32["T"] - r64["T"]) / np.linalg.norm(r64["T"]))
        line["fp64"] = {"value": value64, "ms_per_step": ms64 / K,
                        "achieved_gbs": ach64, "algorithmic_bytes_per_cell_per_launch": b64,
                        "term_ms_avg": r64["t_terms_ms"] / max(r64["n_terms"], 1),
                        "degrees_per_step": [s[1:] if s[0] == 1 else s for s in r64["degrees"]]}
        line["speedup_fp32_bulk_vs_fp64"] = ms64 / ms
        line["rel_l2_fp32_bulk_vs_fp64"] = rel
        # the same steps with the fast (midpoint-candidate) Leja points
        rf = run_gpu(E, torch, wl, "fp32_bulk", K, Wu, dev, world, points="fast")
        msf, valuef = aggregate(rf["ms"], N, K, world, dev)
        line["leja_fast_fp32_bulk"] = {
            "value": valuef, "ms_per_step": msf / K,
            "terms_per_step": float(np.mean([sum(s[1:]) for s in rf["degrees"]])),
            "terms_per_step_exact_points": float(np.mean([sum(s[1:]) for s in r32["degrees"]])),
            "rel_l2_vs_exact_points": float(np.linalg.norm(rf["T"] - r32["T"]) / np.linalg.norm(r32["T"]))}
        rfo = run_forced(E, torch, wl, K, Wu, dev)
        msfo, valuefo = aggregate(rfo["ms"], N, K, world, dev)
        line["forced_fp32_bulk"] = {
            "value": valuefo, "ms_per_step": msfo / K, "inflow": "T_in(t) = 60 + 20 sin(2 pi t)",
            "phi1_terms_per_step": rfo["phi1_terms_per_step"],
            "phi2_terms_per_step": rfo["phi2_terms_per_step"]}
        if not args.no_krylov:
            rk = run_krylov(E, torch, wl, K, Wu, dev)
            msk, valuek = aggregate(rk["ms"], N, K, world, dev)
            line["krylov_fp64"] = {
                "value": valuek, "ms_per_step": msk / K, "m": 10,
                "substeps_per_step": rk["substeps_per_step"], "rejections": rk["rejections"],
                "launches": rk["launches"],
                "rel_l2_vs_leja_fp64": float(np.linalg.norm(rk["T"] - r64["T"]) / np.linalg.norm(r64["T"]))}
    if not args.no_e2e:
        sec = run_e2e(E, torch, wl, K, Wu, dev)
        sec = max_over_ranks(sec, world, dev)
        line["e2e"] = {"value": world * N * K / sec / 1e6, "unit": UNIT,
                       "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sec, ncell, desc = time_oracle(wl, args.slab, args.cpu_steps)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                                "sample": f"{args.cpu_steps} oracle EREM steps on the {desc} "
                                          f"({sec:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the 1024^2 coupled workload: per step, the steady pressure at T^n (warm
# started CG, FP64), then one heat step (EREM FP32-bulk / FP64, or ROS2)
# ---------------------------------------------------------------------------
def run_coupled(E, torch, wl, scheme, precision, steps, warmup, dev):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    import workloads as W

    ctx = E.Context(2, wl.nx, wl.ny, 1, physics=E.Physics(1.0, 1.0, wl.head_drop, 0.0,
                                                         wl.T_inflow, 1), precision=precision)
    lnk, phi, lam = t(wl.lnk), t(wl.phi), t(wl.lam)
    T = t(wl.T0)
    p = t(linear_head(wl.n, wl.nx, wl.head_drop, 0.0))
    if scheme == "erem_from_last":  # each step starts at the last step's substep count
        ctx.set_substep_start(E.EREM_SUBSTEPS_FROM_LAST)
        scheme = "erem"
    st = ctx.pressure_solve(lnk, T, p, tol=1e-10, maxit=200000)
    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), st.flux_in / 1.0)
    ctx.set_physics(E.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 1))
    opts = E.leja_opts(tol=wl.tol, time_terms=True)
    stream = torch.cuda.current_stream()
    T_p = T.clone()  # the temperature p was solved at

    def step():
        if scheme == "strang":
            st, s1 = ctx.coupled_step(T, p, lnk, phi, lam, wl.dt, E.EREM_SPLIT_STRANG,
                                      pressure_tol=1e-10, opts=[opts, opts], T_p=T_p)
            s1.launches += st[0].launches + st[1].launches
            st[1].degree_total += st[0].degree_total
            return s1, st[1]
        s1 = ctx.pressure_solve(lnk, T, p, tol=1e-10, maxit=200000)
        if scheme == "erem":
            s2 = ctx.erem_step(T, wl.dt, p, lnk, phi, lam, opts=opts)
        else:
            code = E.EREM_ROS3P if scheme == "ros3p" else E.EREM_ROS2
            s2 = ctx.rosm_step(T, wl.dt, code, p, lnk, phi, lam, lin_tol=1e-10, maxit=20000)
        return s1, s2

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    cg_it, lin_it, degrees, launches = [], [], [], 0
    e0.record(stream)
    for _ in range(steps):
        s1, s2 = step()
        cg_it.append(s1.lin_iters)
        lin_it.append(s2.lin_iters)
        degrees.append(s2.degree_total)
        launches += s1.launches + s2.launches
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"ms": e0.elapsed_time(e1), "cg_iters_per_step": float(np.mean(cg_it)),
           "stage_iters_per_step": float(np.mean(lin_it)),
           "leja_terms_per_step": float(np.mean(degrees)), "launches": launches,
           "T": T.cpu().numpy(), "rhoc": rc}
    ctx.close()
    return out


def main_coupled(args):
    import torch

    import paper_1209_5553_gb300 as E
    import workloads as W

    rank, world, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init(world, "nccl")
    n = 1024 if args.n == 256 else args.n
    wl = W.coupled2d(n)
    K, Wu = args.steps, args.warmup
    runs = {}
    arms = (("erem_fp32_bulk", "erem", "fp32_bulk"), ("erem_fp64", "erem", "fp64"),
            ("ros2_fp64", "ros2", "fp64"), ("ros3p_fp64", "ros3p", "fp64"),
            ("erem_strang_fp32_bulk", "strang", "fp32_bulk"),
            ("erem_from_last_fp32_bulk", "erem_from_last", "fp32_bulk"))
    want = None if args.arms == "all" else set(args.arms.split(",")) | {"erem_fp32_bulk"}
    for key, scheme, prec in arms:
        if want is not None and key not in want:
            continue
        r = run_coupled(E, torch, wl, scheme, prec, K, Wu, dev)
        ms, value = aggregate(r["ms"], wl.n, K, world, dev)
        r.update(ms=ms, value=value)
        runs[key] = r
    h = runs["erem_fp32_bulk"]
    ref = runs["erem_fp64"]["T"] if "erem_fp64" in runs else h["T"]
    line = {
        "metric": "coupled pressure/temperature Mcell-steps/s (per-step FP64 CG pressure + EREM heat step)",
        "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wu,
        "ms_per_step": h["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"coupled2d_{n}", "grid": [n, n], "cells": wl.n, "dt": wl.dt,
                   "tol": wl.tol, "fluid_model": 1, "pressure_tol": 1e-10,
                   "l2": "working set fits L2 (about 100 MB): L2-resident workload"},
        "gpu_launches": h["launches"],
        "arms": {k: {"value": r["value"], "ms_per_step": r["ms"] / K,
                     "cg_iters_per_step": r["cg_iters_per_step"],
                     "stage_iters_per_step": r["stage_iters_per_step"],
                     "leja_terms_per_step": r["leja_terms_per_step"],
                     "rel_l2_vs_erem_fp64": float(np.linalg.norm(r["T"] - ref) / np.linalg.norm(ref))}
                 for k, r in runs.items()},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the batched ensemble: 512 independent 2D members (n ~ U{64..512}, sigma of
# ln K ~ U[0.5, 2.5], Peclet 50, dt = 0.05); one "step" advances every member
# by one EREM step; a run of K steps is one CUDA graph launch
# ---------------------------------------------------------------------------
ENS_BYTES_PER_CELL_TERM = {"fp32_bulk": 5 * 4 + 4 + 4 + 16, "fp64": 5 * 8 + 8 + 8 + 16}


def ensemble_inputs(E, torch, dev, members):
    """Member fields, GPU pressure solves and heat capacities (Pe = 50 from
    each member's Darcy inflow), as host arrays."""
    import workloads as W

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    out, cg = [], []
    for e in range(members):
        wl = W.ensemble_member(e, members)
        with E.Context(2, wl.nx, wl.ny, physics=E.Physics(1.0, 1.0, wl.head_drop, 0.0,
                                                            wl.T_inflow, 0)) as ctx:
            p = t(linear_head(wl.n, wl.nx, wl.head_drop, 0.0))
            st = ctx.pressure_solve(t(wl.lnk), None, p, tol=1e-10, maxit=200000)
        rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), st.flux_in / 1.0)
        out.append((wl, p.cpu().numpy(), E.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 0)))
        cg.append(st.lin_iters)
    return out, cg


def make_ensemble(E, inputs, precision, tol):
    ens = E.Ensemble([(wl.nx, wl.ny, ph) for wl, _, ph in inputs], precision)
    ens.configure(E.leja_opts(tol=tol), policy=E.EREM_ENS_KEEP_SUBSTEPS)
    for e, (wl, p, _) in enumerate(inputs):
        ens.set_member(e, wl.T0, p, wl.lnk, wl.phi, wl.lam, wl.dt)
    return ens


def run_ensemble(E, torch, inputs, precision, steps, warmup, dev, sample_clocks=False):
    tol = inputs[0][0].tol
    ens = make_ensemble(E, inputs, precision, tol)
    t_tune = time.perf_counter()
    ens.autotune(1)
    t_tune = time.perf_counter() - t_tune
    if warmup:
        ens.run(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(dev.index if dev.index is not None else 0) if sample_clocks else None
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rs = ens.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    stats = [ens.member_stats(e) for e in range(len(inputs))]
    T = [np.zeros(n) for n in ens.sizes]
    for e in range(len(inputs)):
        ens.get_member(e, T[e])
    out = {"ms": ms, "run_ms": rs.t_ms, "iterations": rs.iterations, "cells": rs.cells,
           "cell_terms": rs.cell_terms, "cell_passes": rs.cell_passes, "tile_vecs": rs.tile_vecs,
           "grid": rs.grid, "clocks": clocks, "T": T, "tune_s": t_tune,
           "terms": [s.terms for s in stats], "substeps": [s.substeps for s in stats],
           "failed": rs.members_failed, "ens": ens}
    return out


def ensemble_e2e(E, torch, ens, inputs, steps):
    """One run through the public API with host buffers: every member's T is
    copied in from pinned host memory before the run and read back after."""
    Th = [torch.from_numpy(np.ascontiguousarray(wl.T0)).pin_memory() for wl, _, _ in inputs]
    for e in range(len(inputs)):
        ens.set_temperature(e, Th[e])
    torch.cuda.synchronize()
    t = time.perf_counter()
    for e in range(len(inputs)):
        ens.set_temperature(e, Th[e])
    ens.run(steps)
    for e in range(len(inputs)):
        ens.get_member(e, Th[e])
    torch.cuda.synchronize()
    return time.perf_counter() - t, 8 * sum(ens.sizes)


def time_oracle_ensemble(members, n_sample):
    """The oracle on a bounded sample: one EREM step of each of n_sample
    members spread over the size range (the oracle's own pressure and Peclet
    scaling, outside the timing)."""
    from oracle import fv, timestep as ts
    from oracle.leja import LejaOptions
    import workloads as W

    sizes, _ = W.ensemble_sizes(members)
    order = np.argsort(sizes)
    picks = [int(order[int(q * (members - 1))]) for q in np.linspace(0.1, 0.9, max(n_sample, 1))]
    sec, cells = 0.0, 0
    for e in picks:
        wl = W.ensemble_member(e, members)
        g = fv.Grid(2, wl.nx, wl.ny)
        base = fv.Physics(head_left=wl.head_drop, head_right=0.0, T_inflow=wl.T_inflow)
        p = ts.pressure_solve_direct(g, base, wl.lnk, wl.T0)
        vx = fv.darcy_fluxes(g, base, wl.lnk, p, wl.T0)[0]
        rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), vx[:, :, 0].sum())
        prob = ts.heat_problem(g, fv.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 0),
                               wl.lnk, wl.phi, wl.lam, p)
        t = time.perf_counter()
        ts.erem_step(prob, wl.T0, wl.dt, LejaOptions(tol_a=wl.tol, tol_r=wl.tol))
        sec += time.perf_counter() - t
        cells += wl.n
    desc = (f"one oracle EREM step of each of {len(picks)} members (n = "
            f"{', '.join(str(int(sizes[e])) for e in picks)}) of the {members}-member ensemble")
    return cells / sec / 1e6, sec, desc


def main_ensemble(args):
    import torch

    import paper_1209_5553_gb300 as E

    rank, world, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init(world, "nccl")
    K, Wu = args.steps, args.warmup
    t_in = time.perf_counter()
    inputs, cg = ensemble_inputs(E, torch, dev, args.members)
    t_in = time.perf_counter() - t_in
    cells = sum(wl.n for wl, _, _ in inputs)
    r32 = run_ensemble(E, torch, inputs, "fp32_bulk", K, Wu, dev, sample_clocks=(rank == 0))
    ms, value = aggregate(r32["ms"], cells, K, world, dev)
    peak, peak_kind = measured_peaks()
    b32 = ENS_BYTES_PER_CELL_TERM["fp32_bulk"]
    achieved = b32 * r32["cell_terms"] / (r32["run_ms"] / 1e3) / 1e9
    line = {
        "metric": "ensemble EREM Mcell-steps/s (512 independent 2D members, 64^2..512^2, FP32-bulk)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wu,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"ensemble2d_{args.members}", "members": args.members, "cells": cells,
                   "sizes": "n ~ U{64..512} (seeded), sigma ~ U[0.5, 2.5], Pe 50, dt 0.05, tol 1e-6",
                   "substep_policy": "keep (autotuned start)", "tile_vecs": r32["tile_vecs"],
                   "grid": r32["grid"],
                   "l2": "aggregate sweep 2.3 GB per term (> L2); tail iterations with few "
                         "active members can be L2-resident",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": r32["clocks"],
        "gpu_launches": r32["iterations"],
        "ensemble": {"iterations": r32["iterations"], "graph_launches": 1,
                     "cell_terms": r32["cell_terms"], "cell_passes": r32["cell_passes"],
                     "terms_per_member_run": {"min": int(min(r32["terms"])),
                                              "median": float(np.median(r32["terms"])),
                                              "max": int(max(r32["terms"]))},
                     "substeps_hist": {str(s): r32["substeps"].count(s) for s in sorted(set(r32["substeps"]))},
                     "failed": r32["failed"], "autotune_s": r32["tune_s"], "inputs_s": t_in,
                     "pressure_cg_iters": {"median": float(np.median(cg)), "max": int(max(cg))}},
        "roofline": {"kernel": f"k_ens_iter<float,4,{r32['tile_vecs']}>", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_cell_term": b32,
                     "note": "Leja-term bytes only over the whole run (the other passes, about "
                             f"{100 * r32['cell_passes'] / max(r32['cell_terms'], 1):.1f}% of the "
                             "cell passes, are not counted): a lower bound"},
    }
    if not args.no_fp64:
        r64 = run_ensemble(E, torch, inputs, "fp64", K, Wu, dev)
        ms64, value64 = aggregate(r64["ms"], cells, K, world, dev)
        num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(r32["T"], r64["T"]))
        den = sum(float(np.sum(b ** 2)) for b in r64["T"])
        line["fp64"] = {"value": value64, "ms_per_step": ms64 / K, "tile_vecs": r64["tile_vecs"],
                        "achieved_gbs": ENS_BYTES_PER_CELL_TERM["fp64"] * r64["cell_terms"]
                        / (r64["run_ms"] / 1e3) / 1e9}
        line["speedup_fp32_bulk_vs_fp64"] = ms64 / ms
        line["rel_l2_fp32_bulk_vs_fp64"] = float(np.sqrt(num / den))
        r64["ens"].close()
    if not args.no_e2e:
        sec, nbytes = ensemble_e2e(E, torch, r32["ens"], inputs, K)
        sec = max_over_ranks(sec, world, dev)
        line["e2e"] = {"value": world * cells * K / sec / 1e6, "unit": UNIT,
                       "h2d_bytes_per_step": nbytes / K, "d2h_bytes_per_step": nbytes / K}
    r32["ens"].close()
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sec, desc = time_oracle_ensemble(args.members, args.cpu_steps)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                                "sample": f"{desc} ({sec:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the adjoint workload: 128^3 channels, 60 steps, gradient of a 16-cell misfit
# with respect to ln K and T0 (forward + checkpointed adjoint, FP32-bulk)
# ---------------------------------------------------------------------------
def main_adjoint(args):
    import torch

    import paper_1209_5553_gb300 as E
    import workloads as W
    from paper_1209_5553_gb300.autograd import MisfitModel, misfit

    rank, world, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init(world, "nccl")
    n = 128 if args.n == 256 else args.n
    wl, obs, data = W.adjoint3d(n)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    # heads for a largest face speed of 1 and (rho c) for Pe 1e3, from a GPU pressure solve
    with E.Context(3, n, n, n, physics=E.Physics(1.0, 1.0, wl.head_drop, 0.0, wl.T_inflow, 0)) as ctx:
        st = ctx.pressure_solve(t(wl.lnk), None, t(linear_head(wl.n, wl.nx, wl.head_drop, 0.0)),
                                tol=1e-10, maxit=200000)
    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), 1.0)
    phys = E.Physics(rc, rc, wl.head_drop / st.vmax, 0.0, wl.T_inflow, 0)
    K, Wu = args.steps, args.warmup
    runs = {}
    arms = [("fp32_bulk", "segment"), ("fp32_bulk", "full")]
    if not args.no_fp64:
        arms.append(("fp64", "segment"))
    for prec, tape in arms:
        m = MisfitModel(3, n, n, n, phys, t(wl.phi), t(wl.lam), wl.dt, wl.steps, t(obs, torch.int64),
                        t(data), precision=prec, checkpoint=10, tape=tape)
        lnk0, T00 = t(wl.lnk), t(wl.T0)

        def grad():
            lnk = lnk0.clone().requires_grad_(True)
            T0 = T00.clone().requires_grad_(True)
            L = misfit(lnk, T0, m)
            L.backward()
            return L.detach(), lnk.grad, T0.grad

        for _ in range(Wu):
            grad()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        for _ in range(K):
            L, gl, gt = grad()
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        terms = sum(s[0] and sum(s[1:]) for s in m.schedules)
        runs[prec if tape == "segment" else prec + "_full_tape"] = {"ms_per_gradient": ms, "L": float(L), "glnk": gl.cpu().numpy(),
                      "gT0": gt.cpu().numpy(), "leja_terms_per_run": terms}
        m.close()
    r = runs["fp32_bulk"]
    cell_steps = wl.n * wl.steps
    line = {
        "metric": "adjoint gradient: forward + checkpointed adjoint Mcell-steps/s (128^3, 60 steps, FP32-bulk)",
        "value": cell_steps / (r["ms_per_gradient"] / 1e3) / 1e6, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": Wu, "ms_per_step": r["ms_per_gradient"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"adjoint3d_{n}", "cells": wl.n, "erem_steps": wl.steps,
                   "observations": int(obs.size), "checkpoint_every": 10, "dt": wl.dt,
                   "a 'step' here": "one gradient evaluation (forward run + adjoint run)"},
        "adjoint": {"ms_per_gradient": r["ms_per_gradient"], "misfit": r["L"],
                    "leja_terms_per_forward": r["leja_terms_per_run"]},
    }
    f = runs["fp32_bulk_full_tape"]
    line["adjoint"]["full_tape_ms_per_gradient"] = f["ms_per_gradient"]
    line["adjoint"]["rel_l2_glnk_full_tape_vs_checkpointed"] = float(
        np.linalg.norm(f["glnk"] - r["glnk"]) / np.linalg.norm(r["glnk"]))
    if "fp64" in runs:
        q = runs["fp64"]
        line["adjoint"]["fp64_ms_per_gradient"] = q["ms_per_gradient"]
        line["adjoint"]["rel_l2_glnk_fp32_vs_fp64"] = float(np.linalg.norm(r["glnk"] - q["glnk"]) / np.linalg.norm(q["glnk"]))
        line["adjoint"]["rel_l2_gT0_fp32_vs_fp64"] = float(np.linalg.norm(r["gT0"] - q["gT0"]) / np.linalg.norm(q["gT0"]))
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse_args()
    if a.impl == "reference":
        main_reference(a)
    elif a.workload == "coupled2d":
        main_coupled(a)
    elif a.workload == "ensemble":
        main_ensemble(a)
    elif a.workload == "adjoint":
        main_adjoint(a)
    else:
        main(a)
