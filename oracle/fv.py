"""Cell-centred finite-volume discretization of the equilibrium heat model (oracle).

TEST INFRASTRUCTURE ONLY. This module is part of the CPU oracle that the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use to check the
CUDA path. The product never imports it.

What it follows (Tambue, Berre, Nordbotten, arXiv 1209.5553):

* Model: the heat equation of §2 (eq. ``heat``) in its local-equilibrium limit
  (he -> infinity, so T_s = T_f = T, stated at the end of §2), with one
  volumetric capacity C = phi (rho c)_f + (1 - phi) (rho c)_s and one effective
  conductivity lambda per cell; Darcy's law (eq. ``darcy``, gravity dropped) and
  the steady mass balance for the pressure (the paper's initial state is the
  steady pressure, §5).
* Space discretization (§3.1): control volumes on a structured grid, two-point
  flux approximation with the harmonic transmissibility
  tau_sigma = |sigma| k_i k_j / (k_i d_i + k_j d_j) on interior faces and
  |sigma| k_i / d_i on Dirichlet faces, and standard upwind weighting of the
  advective quantity X on every face.

Everything here is written face by face, as the finite-volume sums over
sigma in E_i are written in §3.1: each face computes one flux and hands it,
with opposite signs, to the two cells it separates.  The Jacobian of the heat
right-hand side is assembled entry by entry as the derivative of those face
fluxes (eq. ``linear``: J_n = D_T G(T^n, p^n)).

Readings of the paper taken here:

* Conductive face flux into cell i is +tau_sigma (T_j - T_i) (the printed
  minus sign in §3.1 is the outward flux).
* Boundary set-up of the synthetic workloads: at x = 0 a Dirichlet pressure
  ``head_left`` and a Dirichlet temperature ``T_inflow`` (conduction through the
  half cell, and the inflow value for upwinding); at x = 1 a Dirichlet pressure
  ``head_right`` and an outflow face that carries X of the boundary cell and no
  conduction; every other boundary face is closed (no flow, no heat flux).
* fluid_model = 1: rho_hat(T) = 1 - 3e-4 (T - 20) and
  mu_hat(T) = exp(-0.02 (T - 20)) (the fluid laws of the 1024^2 workload, divided
  by their reference values).  The pressure equation uses the mass mobility
  K rho_hat / mu_hat, the Darcy flux K / mu_hat, and the advected quantity is
  X = rho_hat(T) T.  fluid_model = 0: rho_hat = mu_hat = 1 and X = T.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# grid and physics descriptions
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Grid:
    """Uniform Cartesian grid on [0, lx] x [0, ly] (x [0, lz]); §3.1.

    Cells are numbered x fastest: i = ix + nx * (iy + ny * iz).  In 2D the
    grid has nz = 1 and a unit thickness, and there are no z faces.
    """

    dim: int
    nx: int
    ny: int
    nz: int = 1
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def h(self):
        hz = self.lz / self.nz if self.dim == 3 else 1.0
        return (self.lx / self.nx, self.ly / self.ny, hz)

    @property
    def volume(self) -> float:
        """|Omega_i|, the same for every cell."""
        hx, hy, hz = self.h
        return hx * hy * hz

    @property
    def face_area(self):
        """|sigma| for faces normal to x, y and z."""
        hx, hy, hz = self.h
        return (hy * hz, hx * hz, hx * hy)

    def cell_centres_x(self) -> np.ndarray:
        hx = self.h[0]
        x = (np.arange(self.nx) + 0.5) * hx
        return np.broadcast_to(x, self.shape).reshape(-1)


@dataclass(frozen=True)
class Physics:
    """Constants of the equilibrium heat model and of its boundary set-up."""

    rhoc_f: float = 1.0
    rhoc_s: float = 1.0
    head_left: float = 1.0
    head_right: float = 0.0
    T_inflow: float = 80.0
    fluid_model: int = 0


# --------------------------------------------------------------------------
# fluid laws (fluid_model = 1 reading of the 1024^2 workload)
# --------------------------------------------------------------------------
def rho_hat(T, phys: Physics):
    if phys.fluid_model == 1:
        return 1.0 - 3e-4 * (T - 20.0)
    return np.ones_like(T)


def mu_hat(T, phys: Physics):
    if phys.fluid_model == 1:
        return np.exp(-0.02 * (T - 20.0))
    return np.ones_like(T)


def advected(T, phys: Physics):
    """X(T): the quantity carried by the Darcy flux (X = rho_f c_pf T_f in §3.1,
    with (rho c)_f factored into the face flux)."""
    return rho_hat(T, phys) * T


def advected_dT(T, phys: Physics):
    """dX/dT, needed for the Jacobian when X is nonlinear in T."""
    if phys.fluid_model == 1:
        return rho_hat(T, phys) + (-3e-4) * T
    return np.ones_like(T)


# --------------------------------------------------------------------------
# face enumeration
# --------------------------------------------------------------------------
def interior_faces(g: Grid):
    """Yield (axis, left_cells, right_cells) for every interior face family.

    ``left`` is the cell on the minus side of the face, ``right`` the cell on
    the plus side; both are flat cell indices (numpy arrays).
    """
    idx = np.arange(g.n).reshape(g.shape)
    yield 0, idx[:, :, :-1].reshape(-1), idx[:, :, 1:].reshape(-1)
    yield 1, idx[:, :-1, :].reshape(-1), idx[:, 1:, :].reshape(-1)
    if g.dim == 3:
        yield 2, idx[:-1, :, :].reshape(-1), idx[1:, :, :].reshape(-1)


def boundary_cells_x(g: Grid):
    """Cells touching the x = 0 face and the x = 1 face (flat indices)."""
    idx = np.arange(g.n).reshape(g.shape)
    return idx[:, :, 0].reshape(-1), idx[:, :, -1].reshape(-1)


def tpfa_interior(k_left, k_right, area, d_left, d_right):
    """Harmonic two-point transmissibility of §3.1:
    tau_sigma = |sigma| k_i k_j / (k_i d_{i,sigma} + k_j d_{j,sigma})."""
    num = area * k_left * k_right
    den = k_left * d_left + k_right * d_right
    out = np.zeros_like(num)
    nz = den != 0
    out[nz] = num[nz] / den[nz]
    return out


def tpfa_dirichlet(k_cell, area, d_cell):
    """Dirichlet-face transmissibility of §3.1: |sigma| k_i / d_{i,sigma}."""
    return area * k_cell / d_cell


# --------------------------------------------------------------------------
# pressure (steady mass balance, eq. masscon4 without storage)
# --------------------------------------------------------------------------
def pressure_system(g: Grid, phys: Physics, lnk, T=None):
    """Assemble the TPFA pressure system A p = b.

    Mass flux out of cell i through face sigma is Upsilon_sigma (p_i - p_sigma)
    with the mass mobility K rho_hat / mu_hat (at T when T is given).  Summing
    the outflow over the faces of each cell and setting it to zero gives a
    symmetric positive definite matrix (Dirichlet faces at x = 0 and x = 1).
    """
    lnk = np.asarray(lnk, dtype=np.float64).reshape(-1)
    Tc = np.full(g.n, 20.0) if T is None else np.asarray(T, np.float64).reshape(-1)
    mob = np.exp(lnk) * rho_hat(Tc, phys) / mu_hat(Tc, phys)
    h = g.h
    area = g.face_area
    rows, cols, vals = [], [], []
    diag = np.zeros(g.n)
    b = np.zeros(g.n)
    for ax, L, R in interior_faces(g):
        ups = tpfa_interior(mob[L], mob[R], area[ax], h[ax] / 2, h[ax] / 2)
        np.add.at(diag, L, ups)
        np.add.at(diag, R, ups)
        rows += [L, R]
        cols += [R, L]
        vals += [-ups, -ups]
    first, last = boundary_cells_x(g)
    for cells, head in ((first, phys.head_left), (last, phys.head_right)):
        ups = tpfa_dirichlet(mob[cells], area[0], h[0] / 2)
        np.add.at(diag, cells, ups)
        np.add.at(b, cells, ups * head)
    rows.append(np.arange(g.n))
    cols.append(np.arange(g.n))
    vals.append(diag)
    A = sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(g.n, g.n),
    )
    A.sum_duplicates()
    return A, b


def linear_head_guess(g: Grid, phys: Physics):
    """Initial guess for the pressure solve: the head interpolated linearly in
    x between the two Dirichlet faces."""
    x = g.cell_centres_x() / g.lx
    return phys.head_left + (phys.head_right - phys.head_left) * x


def darcy_fluxes(g: Grid, phys: Physics, lnk, p, T=None):
    """Volumetric Darcy fluxes v_sigma = int_sigma n . v ds through every face
    (eq. ``darcy`` discretized with TPFA), with the mobility K / mu_hat.

    Returns (vx, vy, vz) on the face arrays of shape (nz, ny, nx+1),
    (nz, ny+1, nx) and (nz+1, ny, nx); each value is the flux in the +axis
    direction.  Closed boundary faces carry zero.
    """
    lnk = np.asarray(lnk, np.float64).reshape(-1)
    p = np.asarray(p, np.float64).reshape(-1)
    Tc = np.full(g.n, 20.0) if T is None else np.asarray(T, np.float64).reshape(-1)
    mob = np.exp(lnk) / mu_hat(Tc, phys)
    h = g.h
    area = g.face_area
    nz, ny, nx = g.shape
    vx = np.zeros((nz, ny, nx + 1))
    vy = np.zeros((nz, ny + 1, nx))
    vz = np.zeros((nz + 1, ny, nx)) if g.dim == 3 else None
    faces = {ax: (L, R) for ax, L, R in interior_faces(g)}
    L, R = faces[0]
    ups = tpfa_interior(mob[L], mob[R], area[0], h[0] / 2, h[0] / 2)
    vx[:, :, 1:-1] = (ups * (p[L] - p[R])).reshape(nz, ny, nx - 1)
    first, last = boundary_cells_x(g)
    ups0 = tpfa_dirichlet(mob[first], area[0], h[0] / 2)
    vx[:, :, 0] = (ups0 * (phys.head_left - p[first])).reshape(nz, ny)
    ups1 = tpfa_dirichlet(mob[last], area[0], h[0] / 2)
    vx[:, :, -1] = (ups1 * (p[last] - phys.head_right)).reshape(nz, ny)
    L, R = faces[1]
    ups = tpfa_interior(mob[L], mob[R], area[1], h[1] / 2, h[1] / 2)
    vy[:, 1:-1, :] = (ups * (p[L] - p[R])).reshape(nz, ny - 1, nx)
    if g.dim == 3:
        L, R = faces[2]
        ups = tpfa_interior(mob[L], mob[R], area[2], h[2] / 2, h[2] / 2)
        vz[1:-1, :, :] = (ups * (p[L] - p[R])).reshape(nz - 1, ny, nx)
    return vx, vy, vz


def cell_net_outflow(g: Grid, vx, vy, vz):
    """Sum over the faces of each cell of the outward volumetric flux
    (discrete divergence of v; zero for a conservative steady flux)."""
    out = vx[:, :, 1:] - vx[:, :, :-1] + vy[:, 1:, :] - vy[:, :-1, :]
    if g.dim == 3:
        out = out + vz[1:, :, :] - vz[:-1, :, :]
    return out.reshape(-1)


# --------------------------------------------------------------------------
# heat right-hand side G(T) and its Jacobian
# --------------------------------------------------------------------------
def capacity(g: Grid, phys: Physics, phi):
    """C_i |Omega_i|, with C = phi (rho c)_f + (1 - phi)(rho c)_s."""
    phi = np.asarray(phi, np.float64).reshape(-1)
    return (phi * phys.rhoc_f + (1.0 - phi) * phys.rhoc_s) * g.volume


def _face_families(g: Grid, vx, vy, vz):
    """Interior faces as (axis, left, right, v) with v the +axis volume flux."""
    for ax, L, R in interior_faces(g):
        if ax == 0:
            v = vx[:, :, 1:-1].reshape(-1)
        elif ax == 1:
            v = vy[:, 1:-1, :].reshape(-1)
        else:
            v = vz[1:-1, :, :].reshape(-1)
        yield ax, L, R, v


def heat_rhs(g: Grid, phys: Physics, phi, lam, T, fluxes):
    """G(T): dT/dt of the semi-discrete heat equation (eq. ``spaceheat2``).

    C_i |Omega_i| dT_i/dt = sum of conductive and advective face fluxes into
    cell i (§3.1).  ``fluxes`` = (vx, vy, vz) from :func:`darcy_fluxes`.
    """
    vx, vy, vz = fluxes
    T = np.asarray(T, np.float64).reshape(-1)
    lam = np.asarray(lam, np.float64).reshape(-1)
    X = advected(T, phys)
    h = g.h
    area = g.face_area
    inflow = np.zeros(g.n)  # heat entering each cell, summed face by face
    for ax, L, R, v in _face_families(g, vx, vy, vz):
        cond = tpfa_interior(lam[L], lam[R], area[ax], h[ax] / 2, h[ax] / 2)
        F = phys.rhoc_f * v
        X_up = np.where(F >= 0, X[L], X[R])
        q = cond * (T[L] - T[R]) + F * X_up  # heat flux in +axis direction
        np.add.at(inflow, L, -q)
        np.add.at(inflow, R, q)
    first, last = boundary_cells_x(g)
    # x = 0: Dirichlet temperature, inflow carries X(T_inflow)
    condD = tpfa_dirichlet(lam[first], area[0], h[0] / 2)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    X_in = advected(np.full(first.shape, phys.T_inflow), phys)
    X_up0 = np.where(F0 > 0, X_in, X[first])
    np.add.at(inflow, first, condD * (phys.T_inflow - T[first]) + F0 * X_up0)
    # x = 1: outflow face carries X of the boundary cell, no conduction
    F1 = phys.rhoc_f * vx[:, :, -1].reshape(-1)
    np.add.at(inflow, last, -F1 * X[last])
    return inflow / capacity(g, phys, phi)


def boundary_heat_inflow(g: Grid, phys: Physics, lam, T, fluxes):
    """Net heat entering the domain through its boundary faces (the only
    non-cancelling terms of sum_i C_i |Omega_i| G_i)."""
    vx, _, _ = fluxes
    T = np.asarray(T, np.float64).reshape(-1)
    lam = np.asarray(lam, np.float64).reshape(-1)
    X = advected(T, phys)
    first, last = boundary_cells_x(g)
    h = g.h
    condD = tpfa_dirichlet(lam[first], g.face_area[0], h[0] / 2)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    X_in = advected(np.full(first.shape, phys.T_inflow), phys)
    q0 = condD * (phys.T_inflow - T[first]) + F0 * np.where(F0 > 0, X_in, X[first])
    F1 = phys.rhoc_f * vx[:, :, -1].reshape(-1)
    return q0.sum() - (F1 * X[last]).sum()


def heat_jacobian(g: Grid, phys: Physics, phi, lam, T, fluxes):
    """J = D_T G(T) (eq. ``linear``), assembled from the derivative of every
    face flux with respect to the temperatures of the cells it touches.
    Returns a scipy CSR matrix (5 or 7 entries per row)."""
    vx, vy, vz = fluxes
    T = np.asarray(T, np.float64).reshape(-1)
    lam = np.asarray(lam, np.float64).reshape(-1)
    dX = advected_dT(T, phys)
    h = g.h
    area = g.face_area
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for ax, L, R, v in _face_families(g, vx, vy, vz):
        cond = tpfa_interior(lam[L], lam[R], area[ax], h[ax] / 2, h[ax] / 2)
        F = phys.rhoc_f * v
        dq_dL = cond + np.where(F >= 0, F * dX[L], 0.0)
        dq_dR = -cond + np.where(F >= 0, 0.0, F * dX[R])
        # inflow[L] -= q ; inflow[R] += q
        add(L, L, -dq_dL)
        add(L, R, -dq_dR)
        add(R, L, dq_dL)
        add(R, R, dq_dR)
    first, last = boundary_cells_x(g)
    condD = tpfa_dirichlet(lam[first], area[0], h[0] / 2)
    F0 = phys.rhoc_f * vx[:, :, 0].reshape(-1)
    add(first, first, -condD + np.where(F0 > 0, 0.0, F0 * dX[first]))
    F1 = phys.rhoc_f * vx[:, :, -1].reshape(-1)
    add(last, last, -F1 * dX[last])
    J = sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(g.n, g.n),
    )
    J.sum_duplicates()
    inv_cap = 1.0 / capacity(g, phys, phi)
    return (sp.diags(inv_cap) @ J).tocsr()
