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
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EREM Mcell-steps/s at 256³ FP32-bulk vs FP64 at ≤1e-5 rel err; HBM GB/s vs peak"
UNIT = "Mcell-steps/s"
# algorithmic bytes per cell of one Leja term (3D): the coefficients of the
# Leja copy of J (7 with the diagonal; 6 when the library keeps the couplings
# only, ctx.leja_coefficients), q read, q written, P read and written
# (FP64).  The running sum is updated at odd m only (both products of a pair
# are in registers then): odd terms move these bytes, even terms 16 fewer.
P_BYTES = 16


def leja_term_bytes(precision: str, ncoef: int) -> int:
    """Odd-term bytes per cell for a Leja copy of ncoef coefficient arrays."""
    esz = 4 if precision == "fp32_bulk" else 8
    return ncoef * esz + 2 * esz + P_BYTES


def term_bytes_per_cell(full_bytes: int, degrees, lagged: bool = False) -> float:
    """Algorithmic bytes per cell of all Leja terms of substeps with these
    degrees: the odd terms (which update P) move full_bytes, the even ones
    full_bytes - 16; in the lagged form of small grids every term updates P
    and moves full_bytes."""
    total = 0
    for m in degrees:
        odd = m if lagged else (m + 1) // 2
        total += odd * full_bytes + (m - odd) * (full_bytes - P_BYTES)
    return float(total)
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
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the FP64 oracle's full-size first step (about a minute on the host)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the coupled 1024^2, ensemble and adjoint sub-objects of the default line")
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
                         "ros3p_fp64, erem_strang_fp32_bulk, erem_from_last_fp32_bulk, and the "
                         "opt-in ros2_adaptive_fp64 (the line needs erem_fp32_bulk); adjoint: subset of fp32_full_tape, fp64 (the "
                         "checkpointed FP32-bulk arm always runs)")
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
    device helpers and the k_leja_term body and entry points."""
    csrc = os.path.join(ROOT, "paper_1209_5553_gb300", "csrc")
    kern = open(os.path.join(csrc, "kernels.cu")).read()
    start = kern.index("__device__ __forceinline__ void leja_term_body(")
    end = kern.index("\n}\n", kern.index("k_leja_term1(const Tq* __restrict__ qi", start))
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


def run_gpu(E, torch, wl, precision, steps, warmup, dev, world, sample_clocks=False, points="exact",
            capture_first=False):
    ctx, T, info = gpu_context(E, torch, wl, precision, dev)
    ctx.set_leja_points(points)
    opts = E.leja_opts(tol=wl.tol, time_terms=True)
    stream = torch.cuda.current_stream()
    first = None
    if capture_first:  # the first step from T^0, untimed, for the oracle check
        st = ctx.erem_step(T, wl.dt, opts=opts)
        first = {"T": T.cpu().numpy(), "schedule": st.schedule}
    # the captured step is the first warm-up step, so that every arm ends on
    # the same state and the cross-arm differences compare the same steps
    for _ in range(warmup - (1 if first is not None else 0)):
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
        lagged = bool(st.terms_lagged)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    barrier(world)
    out = {"ms": ms, "degrees": degrees, "t_terms_ms": t_terms, "n_terms": n_terms,
           "n_leja": n_leja, "launches": launches, "T": T.cpu().numpy(), "clocks": clocks, "info": info,
           "alpha": st.alpha, "beta": st.beta, "first": first, "leja_coefs": ctx.leja_coefficients,
           "lagged": lagged}
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
# CPU oracle: z slabs of the workload (each an independent problem with its
# own pressure solve and velocity scaling) and the full-size first step
# ---------------------------------------------------------------------------
def oracle_slab(wl, z0, nz_s):
    """The oracle's heat problem on planes z0 .. z0+nz_s-1 of the workload
    (the whole workload when nz_s = nz): its own pressure (Jacobi CG from the
    linear head, where the channel family's head is exact), velocity scaled
    to a largest face speed of 1, (rho c) for the Peclet number."""
    from oracle import fv, timestep as ts
    import workloads as W

    n = wl.nx
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
    return prob, f(wl.T0), g.n


def _oracle_slab_worker(n, z0, nz_s, steps, warmup, barrier, queue):
    """One process of the all-core baseline: set up its slab, wait for the
    others, then time `steps` oracle EREM steps."""
    try:
        from oracle import timestep as ts
        from oracle.leja import LejaOptions

        wl = make_workload(n)
        prob, T, ncell = oracle_slab(wl, z0, nz_s)
        opts = LejaOptions(tol_a=wl.tol, tol_r=wl.tol)
        for _ in range(warmup):
            T, _ = ts.erem_step(prob, T, wl.dt, opts)
        barrier.wait(timeout=1800)
        t = time.perf_counter()
        for _ in range(steps):
            T, _ = ts.erem_step(prob, T, wl.dt, opts)
        queue.put((z0, ncell, time.perf_counter() - t, None))
    except Exception as e:  # noqa: BLE001 -- reported to the parent
        barrier.abort()
        queue.put((z0, 0, 0.0, repr(e)))


def host_info():
    """Host cores, CPU model and architecture of the machine the oracle runs on."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    try:
        nproc = len(os.sched_getaffinity(0))
    except AttributeError:
        nproc = os.cpu_count() or 1
    return {"nproc": nproc, "cpu_model": model or platform.processor() or "unknown",
            "arch": platform.machine()}


def time_oracle_all_cores(wl, steps, warmup=0, workers=None):
    """The oracle as it stands (numpy/scipy, one thread per process) on all
    host cores: one spawned process per z slab of the workload, every slab an
    independent problem; the processes set up, meet at a barrier and time
    their steps together.  Returns (Mcell-steps/s summed over the slabs, wall
    seconds of the slowest, processes, description)."""
    import multiprocessing as mp

    host = host_info()
    workers = workers or max(1, min(host["nproc"], wl.nz // 4))
    nz_s = wl.nz // workers
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"  # inherited by the spawned processes: one thread each
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_slab_worker,
                         args=(wl.nx, k * nz_s, nz_s, steps, warmup, barrier, queue))
             for k in range(workers)]
    try:
        for p in procs:
            p.start()
        res = [queue.get(timeout=3600) for _ in procs]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    errs = [r[3] for r in res if r[3]]
    if errs:
        raise RuntimeError(f"oracle worker failed: {errs[0]}")
    sec = max(r[2] for r in res)
    cells = sum(r[1] for r in res)
    desc = (f"{workers} concurrent processes, one per z-slab {wl.nx}x{wl.ny}x{nz_s} of the "
            f"{wl.nx}^3 workload (planes 0..{workers * nz_s - 1}; each slab its own problem)")
    return cells * steps / sec / 1e6, sec, workers, desc


def time_oracle(wl, nz_s, steps, warmup=0):
    """The oracle on one host thread: `steps` EREM steps on the 16-plane
    slab of the workload that holds the most channels."""
    from oracle import timestep as ts
    from oracle.leja import LejaOptions

    lnk = wl.lnk.reshape(wl.nz, wl.ny, wl.nx)
    chan = np.isclose(lnk, np.log(1e4)).sum(axis=(1, 2))
    z0 = max(range(0, wl.nz - nz_s + 1, nz_s), key=lambda z: chan[z:z + nz_s].sum())
    prob, T, ncell = oracle_slab(wl, z0, nz_s)
    opts = LejaOptions(tol_a=wl.tol, tol_r=wl.tol)
    for _ in range(warmup):
        T, _ = ts.erem_step(prob, T, wl.dt, opts)
    t = time.perf_counter()
    for _ in range(steps):
        T, _ = ts.erem_step(prob, T, wl.dt, opts)
    sec = time.perf_counter() - t
    desc = f"z-slab {wl.nx}x{wl.ny}x{nz_s} (planes {z0}..{z0 + nz_s - 1}) of the {wl.nx}^3 workload"
    return ncell * steps / sec / 1e6, sec, ncell, desc


def oracle_check(wl, firsts):
    """Relative L2 errors of the GPU's first steps from T^0 against one
    oracle EREM step of the whole workload (FP64, same inputs): on the state
    T^1 and on the increment T^1 - T^0 the step computed."""
    from oracle import timestep as ts
    from oracle.leja import LejaOptions

    t = time.perf_counter()
    prob, T0, _ = oracle_slab(wl, 0, wl.nz)
    T1, res = ts.erem_step(prob, T0, wl.dt, LejaOptions(tol_a=wl.tol, tol_r=wl.tol))
    sec = time.perf_counter() - t
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out = {"oracle_schedule": res.schedule, "oracle_s": sec,
           "what": "one step from T^0 of the full workload; relative L2 of the state T^1 and of "
                   "the increment T^1 - T^0 against the FP64 oracle"}
    for key, f in firsts.items():
        if f is None:
            continue
        out[key] = {"rel_l2_state": rel(f["T"], T1), "rel_l2_increment": rel(f["T"] - T0, T1 - T0),
                    "schedule": f["schedule"]}
    return out


# ---------------------------------------------------------------------------
def main_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    wl = make_workload(args.n)
    value, sec, workers, desc = time_oracle_all_cores(wl, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"channels3d_{args.n}", "sample": desc, "dt": wl.dt, "tol": wl.tol},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{args.steps} oracle EREM steps in each of {desc}",
                         "host": host_info()},
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

    check = rank == 0 and world == 1 and not args.no_oracle_check
    r32 = run_gpu(E, torch, wl, "fp32_bulk", K, Wu, dev, world, sample_clocks=(rank == 0),
                  capture_first=check)
    ms, value = aggregate(r32["ms"], N, K, world, dev)
    peak, peak_kind = measured_peaks()
    b32 = leja_term_bytes("fp32_bulk", r32["leja_coefs"])
    # a Leja term moves the coefficients once and q in and out; the odd terms
    # also read and write P: 48 B per cell for odd m, 32 B for even m with the
    # couplings-only copy (52 and 36 with the diagonal)
    sec_leja = r32["t_terms_ms"] / 1e3
    bpc = term_bytes_per_cell(b32, [m for s in r32["degrees"] for m in s[1:]], r32["lagged"])
    achieved = bpc * N / sec_leja / 1e9 if r32["n_terms"] else None
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
                     "algorithmic_bytes_per_cell_per_launch": bpc / max(r32["n_terms"], 1),
                     "algorithmic_bytes_per_cell": {"odd_terms": b32, "even_terms": b32 - P_BYTES},
                     "launch_ms_avg": r32["t_terms_ms"] / max(r32["n_terms"], 1),
                     "timing": "CUDA events on the launching stream around each chunk of term "
                               "launches (gaps and launches after the stop included: the "
                               "per-term time is an upper bound)",
                     "effective_gbs_at_odd_term_bytes": effective,
                     "term_ms_avg": r32["t_terms_ms"] / max(r32["n_terms"], 1)},
        "setup": r32["info"],
    }
    if not args.no_fp64:
        r64 = run_gpu(E, torch, wl, "fp64", K, Wu, dev, world, capture_first=check)
        ms64, value64 = aggregate(r64["ms"], N, K, world, dev)
        b64 = leja_term_bytes("fp64", r64["leja_coefs"])
        bpc64 = term_bytes_per_cell(b64, [m for s in r64["degrees"] for m in s[1:]], r64["lagged"])
        ach64 = bpc64 * N / (r64["t_terms_ms"] / 1e3) / 1e9 if r64["n_terms"] else None
        rel = float(np.linalg.norm(r32["T"] - r64["T"]) / np.linalg.norm(r64["T"]))
        line["fp64"] = {"value": value64, "ms_per_step": ms64 / K,
                        "achieved_gbs": ach64,
                        "algorithmic_bytes_per_cell_per_launch": bpc64 / max(r64["n_terms"], 1),
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
    if not args.no_extra:
        # the other workloads, each with its own value, step time, dominant
        # kernel's roofline and FP32-bulk/FP64 ratio
        line["coupled2d"] = coupled_summary(E, torch, dev, world, K, Wu, check=check)
        line["ensemble"] = ensemble_summary(E, torch, dev, world, Wu)
        line["adjoint"] = adjoint_summary(E, torch, dev, world)
    if check:
        line["rel_l2_vs_oracle"] = oracle_check(wl, {
            "fp32_bulk": r32["first"], "fp64": r64["first"] if not args.no_fp64 else None})
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sec, workers, desc = time_oracle_all_cores(wl, args.cpu_steps)
        v1, sec1, _, desc1 = time_oracle(wl, args.slab, args.cpu_steps)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
                                "sample": f"{args.cpu_steps} oracle EREM steps in each of {desc} "
                                          f"({sec:.1f} s); the rate is summed over the processes",
                                "host": host_info(),
                                "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                  "sample": f"{args.cpu_steps} oracle EREM steps on the "
                                                            f"{desc1} ({sec1:.1f} s)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the 1024^2 coupled workload: per step, the steady pressure at T^n (warm
# started CG, FP64), then one heat step (EREM FP32-bulk / FP64, or ROS2)
# ---------------------------------------------------------------------------
def run_coupled(E, torch, wl, scheme, precision, steps, warmup, dev, capture_first=False):
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
    ada = {"h0": wl.dt, "accepted": [], "rejected": []}

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
        elif scheme in ("ros2_adaptive", "ros3p_adaptive"):
            # the heat step over dt by embedded-ROS error control (tolerances of
            # the EREM arms), starting from the previous step's longest
            # accepted length
            code = E.EREM_ROS3P if scheme == "ros3p_adaptive" else E.EREM_ROS2
            ctx.set_state(T, p, lnk, phi, lam, wl.dt)
            a, dts = ctx.rosm_integrate(T, wl.dt, ada["h0"], code, wl.tol, wl.tol, lin_tol=1e-10,
                                        maxit=20000)
            ada["h0"] = min(wl.dt, a.dt_max)
            ada["accepted"].append(a.accepted)
            ada["rejected"].append(a.rejected)
            s2 = types.SimpleNamespace(lin_iters=a.lin_iters, degree_total=0, degrees=[],
                                       substeps=0, launches=a.launches, t_terms_ms=0.0,
                                       n_terms_timed=0, terms_lagged=0)
        else:
            code = E.EREM_ROS3P if scheme == "ros3p" else E.EREM_ROS2
            s2 = ctx.rosm_step(T, wl.dt, code, p, lnk, phi, lam, lin_tol=1e-10, maxit=20000)
        return s1, s2

    first = None
    for k in range(warmup):
        _, s2 = step()
        if capture_first and k == 0:  # the first step from T^0 (a warm-up step), for the oracle check
            first = {"T": T.cpu().numpy(), "schedule": s2.schedule}
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    cg_it, lin_it, degrees, launches, t_terms, n_terms, scheds = [], [], [], 0, 0.0, 0, []
    e0.record(stream)
    for _ in range(steps):
        s1, s2 = step()
        cg_it.append(s1.lin_iters)
        lin_it.append(s2.lin_iters)
        degrees.append(s2.degree_total)
        scheds.append(list(s2.degrees[:s2.substeps]))
        launches += s1.launches + s2.launches
        t_terms += s2.t_terms_ms
        n_terms += s2.n_terms_timed
        lagged = bool(s2.terms_lagged)
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"ms": e0.elapsed_time(e1), "cg_iters_per_step": float(np.mean(cg_it)),
           "stage_iters_per_step": float(np.mean(lin_it)),
           "leja_terms_per_step": float(np.mean(degrees)), "launches": launches,
           "leja_coefs": ctx.leja_coefficients, "lagged": lagged,
           "T": T.cpu().numpy(), "rhoc": rc, "t_terms_ms": t_terms, "n_terms": n_terms,
           "degrees": [m for sc in scheds for m in sc], "first": first}
    if ada["accepted"]:
        out["ros_steps_per_step"] = float(np.mean(ada["accepted"][-steps:]))
        out["ros_rejections_per_step"] = float(np.mean(ada["rejected"][-steps:]))
    ctx.close()
    return out


def oracle_coupled_check(wl, rc, firsts):
    """Relative L2 errors of the GPU's first coupled steps from T^0 against
    one oracle sequential step (§3.2: steady pressure at T^0 by a sparse
    direct solve, Darcy fluxes at T^0, one EREM heat step with the
    T-dependent fluid laws; FP64), with the heat capacity the GPU run took
    from its own pressure solve."""
    from oracle import fv, timestep as ts
    from oracle.leja import LejaOptions

    t = time.perf_counter()
    g = fv.Grid(2, wl.nx, wl.ny)
    ph = fv.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 1)
    T0 = wl.T0
    T1, _, res = ts.sequential_step(g, ph, wl.lnk, wl.phi, wl.lam, T0.copy(), None, wl.dt,
                                    opts=LejaOptions(tol_a=wl.tol, tol_r=wl.tol))
    sec = time.perf_counter() - t
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out = {"oracle_schedule": res.schedule, "oracle_s": sec,
           "what": "one coupled step from T^0 (pressure, then the heat step); relative L2 of the "
                   "state T^1 and of the increment T^1 - T^0 against the FP64 oracle",
           "note": "the GPU's pressure is its CG to 1e-10, the oracle's a direct solve: the FP64 "
                   "arm's difference is that of the pressure (with the oracle's pressure the "
                   "parity tests hold 1e-11)"}
    for key, f in firsts.items():
        if f is not None:
            out[key] = {"rel_l2_state": rel(f["T"], T1), "rel_l2_increment": rel(f["T"] - T0, T1 - T0),
                        "schedule": f["schedule"]}
    return out


def coupled_summary(E, torch, dev, world, K, Wu, check=False):
    """The 1024^2 coupled workload for the default line: EREM FP32-bulk and
    FP64 and ROS2 (FP64), K steps each after Wu warm-up steps; with check,
    the first EREM steps against one oracle step."""
    import workloads as W

    wl = W.coupled2d(1024)
    runs = {}
    for key, scheme, prec in (("erem_fp32_bulk", "erem", "fp32_bulk"), ("erem_fp64", "erem", "fp64"),
                              ("ros2_fp64", "ros2", "fp64")):
        r = run_coupled(E, torch, wl, scheme, prec, K, Wu, dev, capture_first=check and scheme == "erem")
        ms, value = aggregate(r["ms"], wl.n, K, world, dev)
        r.update(ms=ms, value=value)
        runs[key] = r
    h, d, q = runs["erem_fp32_bulk"], runs["erem_fp64"], runs["ros2_fp64"]
    peak, kind = measured_peaks()
    b = leja_term_bytes("fp32_bulk", h["leja_coefs"])  # 2D: the copy's coefficients, q in/out, P in/out
    h_lag = h["lagged"]
    bpc = term_bytes_per_cell(b, h["degrees"], h_lag)
    ach = bpc * wl.n / (h["t_terms_ms"] / 1e3) / 1e9 if h["n_terms"] else None
    rel = lambda a, b_: float(np.linalg.norm(a - b_) / np.linalg.norm(b_))
    out = {
        "workload": "coupled2d_1024", "cells": wl.n, "steps": K, "warmup": Wu, "unit": UNIT,
        "value": h["value"], "ms_per_step": h["ms"] / K,
        "what": "per step: steady FP64 pressure CG at T^n (multigrid-preconditioned, to 1e-10), "
                "then one heat step with the T-dependent fluid laws",
        "leja_terms_per_step": h["leja_terms_per_step"], "cg_iters_per_step": h["cg_iters_per_step"],
        "fp64": {"value": d["value"], "ms_per_step": d["ms"] / K},
        "speedup_fp32_bulk_vs_fp64": d["ms"] / h["ms"],
        "rel_l2_fp32_bulk_vs_fp64": rel(h["T"], d["T"]),
        "ros2_fp64": {"value": q["value"], "ms_per_step": q["ms"] / K,
                      "stage_iters_per_step": q["stage_iters_per_step"],
                      "rel_l2_vs_erem_fp64": rel(q["T"], d["T"])},
        "roofline": {"kernel": "k_leja_term<float,4,2>", "bound": "hbm", "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak if ach else None, "traffic": None,
                     "peak_source": f"{kind} hbm_gbs",
                     "algorithmic_bytes_per_cell": {"odd_terms": b,
                                                   "even_terms": b if h_lag else b - P_BYTES},
                     "terms_lagged": h_lag,
                     "term_ms_avg": h["t_terms_ms"] / max(h["n_terms"], 1),
                     "note": "the 1024^2 term's working set (about 50 MB) stays in L2, so the "
                             "achieved rate is not an HBM figure"},
    }
    if check and h["first"] is not None:
        out["rel_l2_vs_oracle"] = oracle_coupled_check(
            wl, h["rhoc"], {"fp32_bulk": h["first"], "fp64": d["first"]})
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
            ("erem_from_last_fp32_bulk", "erem_from_last", "fp32_bulk"),
            ("ros2_adaptive_fp64", "ros2_adaptive", "fp64"))
    opt_in = {"ros2_adaptive_fp64"}  # not part of "all": many short ROS steps per coupled step
    want = None if args.arms == "all" else set(args.arms.split(",")) | {"erem_fp32_bulk"}
    for key, scheme, prec in arms:
        if (want is None and key in opt_in) or (want is not None and key not in want):
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
                     "rel_l2_vs_erem_fp64": float(np.linalg.norm(r["T"] - ref) / np.linalg.norm(ref)),
                     **{q: r[q] for q in ("ros_steps_per_step", "ros_rejections_per_step") if q in r}}
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


def ensemble_term_bytes(prec, r):
    """Algorithmic bytes of the run's Leja terms: per member, cells x terms x
    (its Leja copy's coefficient arrays, q in and out, P in and out)."""
    esz = 4 if prec == "fp32_bulk" else 8
    return sum(n * t * (nc * esz + 2 * esz + P_BYTES)
               for n, t, nc in zip(r["sizes"], r["terms"], r["leja_coefs"]))


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
    ens.autotune(5)  # the cluster size for a run of many steps (a 1-step probe favours large clusters)
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
    out = {"ms": ms, "run_ms": rs.t_ms, "passes": rs.passes, "cells": rs.cells,
           "cell_terms": rs.cell_terms, "cell_passes": rs.cell_passes, "cluster_ctas": rs.cluster_ctas,
           "clusters": rs.clusters, "cta_threads": rs.cta_threads, "clocks": clocks, "T": T,
           "tune_s": t_tune, "graph": rs.graph,
           "terms": [s.terms for s in stats], "substeps": [s.substeps for s in stats],
           "leja_coefs": [s.leja_coefficients for s in stats], "sizes": list(ens.sizes),
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


def ensemble_summary(E, torch, dev, world, Wu, members=512, steps=30):
    """The 512-member ensemble for the default line: one graph launch of the
    workload's 30 EREM steps per precision, after Wu warm-up steps."""
    t_in = time.perf_counter()
    inputs, _ = ensemble_inputs(E, torch, dev, members)
    t_in = time.perf_counter() - t_in
    cells = sum(wl.n for wl, _, _ in inputs)
    peak, kind = measured_peaks()
    out = {"workload": f"ensemble2d_{members}", "members": members, "cells": cells, "steps": steps,
           "warmup": Wu, "unit": UNIT, "inputs_s": t_in}
    Ts = {}
    for prec in ("fp32_bulk", "fp64"):
        r = run_ensemble(E, torch, inputs, prec, steps, Wu, dev)
        ms, value = aggregate(r["ms"], cells, steps, world, dev)
        tb = ensemble_term_bytes(prec, r)
        b = tb / max(r["cell_terms"], 1)
        ach = tb / (r["run_ms"] / 1e3) / 1e9
        Ts[prec] = r["T"]
        summary = {"value": value, "ms_per_step": ms / steps, "member_passes": r["passes"],
                   "cluster_ctas": r["cluster_ctas"], "clusters": r["clusters"],
                   "cuda_graph": bool(r["graph"]), "autotune_s": r["tune_s"],
                   "terms_per_member_run": {"median": float(np.median(r["terms"])),
                                            "max": int(max(r["terms"]))}}
        if prec == "fp32_bulk":
            out.update(summary)
            out["roofline"] = {"kernel": "k_ens_cluster<float,4>", "bound": "hbm",
                               "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                               "traffic": None, "peak_source": f"{kind} hbm_gbs",
                               "algorithmic_bytes_per_cell_term": b,
                               "note": "Leja-term bytes only over the whole run; each member's "
                                       "Leja working set stays in L2 while its cluster runs it, so "
                                       "the rate can exceed the HBM copy bandwidth"}
        else:
            out["fp64"] = summary
            out["speedup_fp32_bulk_vs_fp64"] = summary["ms_per_step"] / out["ms_per_step"]
        r["ens"].close()
    num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(Ts["fp32_bulk"], Ts["fp64"]))
    den = sum(float(np.sum(b ** 2)) for b in Ts["fp64"])
    out["rel_l2_fp32_bulk_vs_fp64"] = float(np.sqrt(num / den))
    return out


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
    tb32 = ensemble_term_bytes("fp32_bulk", r32)
    b32 = tb32 / max(r32["cell_terms"], 1)
    achieved = tb32 / (r32["run_ms"] / 1e3) / 1e9
    line = {
        "metric": "ensemble EREM Mcell-steps/s (512 independent 2D members, 64^2..512^2, FP32-bulk)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wu,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"ensemble2d_{args.members}", "members": args.members, "cells": cells,
                   "sizes": "n ~ U{64..512} (seeded), sigma ~ U[0.5, 2.5], Pe 50, dt 0.05, tol 1e-6",
                   "substep_policy": "keep (autotuned start)", "cluster_ctas": r32["cluster_ctas"],
                   "clusters": r32["clusters"], "cta_threads": r32["cta_threads"],
                   "cuda_graph": bool(r32["graph"]),
                   "l2": "all members 1.9 GB of Leja working set (> L2); one member's (at most "
                         "9.4 MB) stays L2-resident while its cluster runs it",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "clocks": r32["clocks"],
        "gpu_launches": 1,
        "ensemble": {"member_passes": r32["passes"], "kernel_launches": 1,
                     "cell_terms": r32["cell_terms"], "cell_passes": r32["cell_passes"],
                     "terms_per_member_run": {"min": int(min(r32["terms"])),
                                              "median": float(np.median(r32["terms"])),
                                              "max": int(max(r32["terms"]))},
                     "substeps_hist": {str(s): r32["substeps"].count(s) for s in sorted(set(r32["substeps"]))},
                     "failed": r32["failed"], "autotune_s": r32["tune_s"], "inputs_s": t_in,
                     "pressure_cg_iters": {"median": float(np.median(cg)), "max": int(max(cg))}},
        "roofline": {"kernel": "k_ens_cluster<float,4>", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_cell_term": b32,
                     "note": "Leja-term bytes only over the whole run (the other passes, about "
                             f"{100 * r32['cell_passes'] / max(r32['cell_terms'], 1):.1f}% of the "
                             "cell passes, are not counted); each member's Leja working set stays "
                             "in L2 while its cluster runs it, so the rate can exceed the HBM copy "
                             "bandwidth"},
    }
    if not args.no_fp64:
        r64 = run_ensemble(E, torch, inputs, "fp64", K, Wu, dev)
        ms64, value64 = aggregate(r64["ms"], cells, K, world, dev)
        num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(r32["T"], r64["T"]))
        den = sum(float(np.sum(b ** 2)) for b in r64["T"])
        line["fp64"] = {"value": value64, "ms_per_step": ms64 / K, "cluster_ctas": r64["cluster_ctas"],
                        "achieved_gbs": ensemble_term_bytes("fp64", r64)
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
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{desc} ({sec:.1f} s)", "host": host_info()}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the adjoint workload: 128^3 channels, 60 steps, gradient of a 16-cell misfit
# with respect to ln K and T0 (forward + checkpointed adjoint, FP32-bulk)
# ---------------------------------------------------------------------------
def adjoint_setup(E, torch, dev, n):
    import workloads as W

    wl, obs, data = W.adjoint3d(n)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    # heads for a largest face speed of 1 and (rho c) for Pe 1e3, from a GPU pressure solve
    with E.Context(3, n, n, n, physics=E.Physics(1.0, 1.0, wl.head_drop, 0.0, wl.T_inflow, 0)) as ctx:
        st = ctx.pressure_solve(t(wl.lnk), None, t(linear_head(wl.n, wl.nx, wl.head_drop, 0.0)),
                                tol=1e-10, maxit=200000)
    rc = W.rhoc_for_peclet(wl.peclet, float(wl.lam[0]), 1.0)
    phys = E.Physics(rc, rc, wl.head_drop / st.vmax, 0.0, wl.T_inflow, 0)
    return wl, obs, data, phys, t


def adjoint_runs(E, torch, dev, n, K, Wu, arms):
    """K gradient evaluations (after Wu) of the misfit for each (precision,
    tape) arm; returns the workload and per-arm results."""
    from paper_1209_5553_gb300.autograd import MisfitModel, misfit

    wl, obs, data, phys, t = adjoint_setup(E, torch, dev, n)
    runs = {}
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
        runs[prec if tape == "segment" else prec + "_full_tape"] = {
            "ms_per_gradient": ms, "L": float(L), "glnk": gl.cpu().numpy(), "gT0": gt.cpu().numpy(),
            "leja_terms_per_run": terms}
        m.close()
    return wl, obs, phys, t, runs


def adjoint_forward_terms(E, torch, wl, phys, t):
    """The forward run's Leja terms timed on their launching stream: the
    adjoint workload's dominant kernel (k_leja_term<float,4,3> at 128^3)."""
    n = wl.nx
    with E.Context(3, n, n, n, physics=phys, precision="fp32_bulk") as ctx:
        lnk = t(wl.lnk)
        p = t(linear_head(wl.n, wl.nx, phys.head_left, 0.0))
        ctx.pressure_solve(lnk, None, p, tol=1e-12, maxit=200000)
        T = t(wl.T0)
        ctx.set_state(T, p, lnk, t(wl.phi), t(wl.lam), wl.dt)
        opts = E.leja_opts(tol=wl.tol, time_terms=True)
        ms, terms, degrees = 0.0, 0, []
        for _ in range(wl.steps):
            st = ctx.erem_step(T, wl.dt, opts=opts)
            ms += st.t_terms_ms
            terms += st.n_terms_timed
            degrees += list(st.degrees[:st.substeps])
            lagged = bool(st.terms_lagged)
        ncoef = ctx.leja_coefficients
    return ms, terms, degrees, ncoef, lagged


def adjoint_summary(E, torch, dev, world, n=128, K=2, Wu=1):
    """The 128^3 adjoint for the default line: FP32-bulk checkpointed, with
    the full tape, and FP64, K gradients each after Wu."""
    wl, obs, phys, t, runs = adjoint_runs(E, torch, dev, n, K, Wu,
                                          [("fp32_bulk", "segment"), ("fp32_bulk", "full"),
                                           ("fp64", "segment")])
    r, f, q = runs["fp32_bulk"], runs["fp32_bulk_full_tape"], runs["fp64"]
    ms = max_over_ranks(r["ms_per_gradient"], world, dev)
    peak, kind = measured_peaks()
    tms, terms, degrees, ncoef, lagged = adjoint_forward_terms(E, torch, wl, phys, t)
    b = leja_term_bytes("fp32_bulk", ncoef)
    h_lag = lagged
    ach = term_bytes_per_cell(b, degrees, lagged) * wl.n / (tms / 1e3) / 1e9 if terms else None
    rel = lambda a, b_: float(np.linalg.norm(a - b_) / np.linalg.norm(b_))
    return {
        "workload": f"adjoint3d_{n}", "cells": wl.n, "erem_steps": wl.steps, "gradients": K,
        "warmup": Wu, "unit": UNIT, "what": "one gradient = forward run + checkpointed adjoint",
        "value": world * wl.n * wl.steps / (ms / 1e3) / 1e6, "ms_per_gradient": ms,
        "full_tape_ms_per_gradient": f["ms_per_gradient"],
        "fp64": {"ms_per_gradient": q["ms_per_gradient"]},
        "speedup_fp32_bulk_vs_fp64": q["ms_per_gradient"] / r["ms_per_gradient"],
        "rel_l2_glnk_fp32_bulk_vs_fp64": rel(r["glnk"], q["glnk"]),
        "rel_l2_gT0_fp32_bulk_vs_fp64": rel(r["gT0"], q["gT0"]),
        "rel_l2_glnk_full_tape_vs_checkpointed": rel(f["glnk"], r["glnk"]),
        "leja_terms_per_forward": r["leja_terms_per_run"],
        "roofline": {"kernel": "k_leja_term<float,4,3>", "bound": "hbm", "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak if ach else None, "traffic": None,
                     "peak_source": f"{kind} hbm_gbs",
                     "algorithmic_bytes_per_cell": {"odd_terms": b,
                                                   "even_terms": b if h_lag else b - P_BYTES},
                     "terms_lagged": h_lag,
                     "term_ms_avg": tms / max(terms, 1),
                     "note": "timed over a 60-step forward run; a 128^3 term moves 109 MB, "
                             "partly served by the 129 MB L2"},
    }


def main_adjoint(args):
    import torch

    import paper_1209_5553_gb300 as E

    rank, world, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init(world, "nccl")
    n = 128 if args.n == 256 else args.n
    K, Wu = args.steps, args.warmup
    arms = [("fp32_bulk", "segment"), ("fp32_bulk", "full")]
    if not args.no_fp64:
        arms.append(("fp64", "segment"))
    if args.arms != "all":  # fp32_bulk (checkpointed) always runs; fp32_full_tape, fp64 on request
        want = set(args.arms.split(","))
        arms = [a for a in arms if a == ("fp32_bulk", "segment")
                or (a == ("fp32_bulk", "full") and "fp32_full_tape" in want)
                or (a[0] == "fp64" and "fp64" in want)]
    wl, obs, _, _, runs = adjoint_runs(E, torch, dev, n, K, Wu, arms)
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
    if "fp32_bulk_full_tape" in runs:
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
