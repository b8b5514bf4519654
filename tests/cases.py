"""Seeded cases shared by the GPU parity tests and smoke checks.

Every input is built on the oracle side (fields from ``workloads``, pressure
from the oracle's direct solve, Peclet scaling from the oracle's fluxes), and
the same arrays go to the CUDA path.  Nothing here reads a CUDA result.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import workloads as W
from oracle import fv, timestep as ts


@dataclass
class Case:
    grid: fv.Grid
    phys: fv.Physics
    lnk: np.ndarray
    phi: np.ndarray
    lam: np.ndarray
    T0: np.ndarray
    p: np.ndarray
    dt: float
    steps: int

    @property
    def n(self):
        return self.grid.n

    def problem(self, T_visc=None):
        return ts.heat_problem(self.grid, self.phys, self.lnk, self.phi, self.lam, self.p, T_visc)

    def gpu_physics(self):
        import paper_1209_5553_gb300 as E

        ph = self.phys
        return E.Physics(ph.rhoc_f, ph.rhoc_s, ph.head_left, ph.head_right, ph.T_inflow,
                         ph.fluid_model)

    def dims(self):
        g = self.grid
        return (g.dim, g.nx, g.ny, g.nz)


def from_workload(wl: W.Workload, pressure: str = "direct") -> Case:
    g = fv.Grid(wl.dim, wl.nx, wl.ny, wl.nz)
    base = fv.Physics(head_left=wl.head_drop, head_right=0.0, T_inflow=wl.T_inflow,
                      fluid_model=wl.fluid_model)
    if pressure == "direct":
        p = ts.pressure_solve_direct(g, base, wl.lnk, wl.T0)
    else:
        p = ts.pressure_solve_cg(g, base, wl.lnk, wl.T0, tol=1e-13)[0]
    vx, vy, vz = fv.darcy_fluxes(g, base, wl.lnk, p, wl.T0)
    lam0 = float(wl.lam[0])
    if wl.velocity_scale == "max":
        area = g.face_area
        vmax = max(np.abs(vx).max() / area[0], np.abs(vy).max() / area[1],
                   np.abs(vz).max() / area[2] if vz is not None else 0.0)
        p = p / vmax
        base = fv.Physics(head_left=wl.head_drop / vmax, head_right=0.0, T_inflow=wl.T_inflow,
                          fluid_model=wl.fluid_model)
        rc = W.rhoc_for_peclet(wl.peclet, lam0, 1.0)
    else:
        width = g.ly * (g.lz if g.dim == 3 else 1.0)
        U = vx[:, :, 0].sum() / width
        rc = W.rhoc_for_peclet(wl.peclet, lam0, U)
    phys = fv.Physics(rc, rc, base.head_left, base.head_right, wl.T_inflow, wl.fluid_model)
    return Case(g, phys, wl.lnk, wl.phi, wl.lam, wl.T0.copy(), p, wl.dt, wl.steps)


def heat2d(n=64, **kw) -> Case:
    return from_workload(W.heat2d(n, **kw))


def heat2d_rect(nx, ny, **kw) -> Case:
    return from_workload(W.heat2d_rect(nx, ny, **kw))


def channels3d(n, **kw) -> Case:
    return from_workload(W.channels3d(n, **kw))


def coupled2d(n, **kw) -> Case:
    return from_workload(W.coupled2d(n, **kw))


def random_case(dim, nx, ny, nz=1, seed=0, fluid_model=0, pe=30.0) -> Case:
    """Heterogeneous fields of every kind (lambda, phi, capacities differ)."""
    rng = np.random.default_rng(seed)
    g = fv.Grid(dim, nx, ny, nz)
    n = g.n
    lnk = rng.normal(0, 1, n)
    phi = rng.uniform(0.1, 0.35, n)
    lam = rng.uniform(0.5, 3.0, n)
    T0 = rng.uniform(20, 80, n)
    base = fv.Physics(head_left=1.0, head_right=0.0, T_inflow=80.0, fluid_model=fluid_model)
    p = ts.pressure_solve_direct(g, base, lnk, T0)
    phys = fv.Physics(pe, 0.7 * pe, 1.0, 0.0, 80.0, fluid_model)
    return Case(g, phys, lnk, phi, lam, T0, p, 0.02, 3)


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
