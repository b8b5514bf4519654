"""Seeded synthetic inputs for the EREM heat-transport workloads.

This module is shared by the CUDA path's callers (``bench.py``, the GPU tests)
and by the CPU oracle's callers.  It holds no arithmetic of the method: it
only draws fields (log-permeability, porosity, conductivity, initial
temperature) and states the constants of each workload.  Quantities that need
a pressure solution (the Darcy velocity scale used to set the Peclet number)
are computed by each caller with its own pressure solver; the helper
:func:`rhoc_for_peclet` only turns such a velocity into a heat capacity.

The paper's experiments (§5: a 3D two-layer reservoir with wells and a 2D
fractured reservoir) use meshes and well models that are not published, so the
workloads below are synthetic stand-ins with the shapes, sizes and structure
of the five named workloads:

* ``heat2d_64``     2D 64x64, ln k Gaussian (sigma 1, correlation 0.1),
                    phi 0.2, lambda 2.0, T0 20, T_in 80, Pe 50, 20 steps of 0.05
* ``coupled2d_1024`` 2D 1024x1024, ln k Gaussian (sigma 2, correlation 0.02),
                    nonlinear fluid laws, 200 steps of 0.005
* ``channels3d_256`` 3D 256^3, 16 z-layers with ln k ~ N(0, 1) and 8 x-aligned
                    8x8-cell channels with k = 1e4, phi 0.2, lambda 1,
                    max face speed 1, Pe 1e3, 50 steps of 1/32
* ``ensemble2d``    512 2D members, n ~ U{64..512}, sigma ~ U[0.5, 2.5]
* ``channels3d_128`` the 3D family at 128^3 (4x4-cell channels), 60 steps of 1/16

Gaussian fields: squared-exponential covariance exp(-r^2 / (2 l^2)) on the
periodic n^d grid, spectral synthesis from PCG64(seed) white noise, then
shifted and scaled to sample mean 0 and sample standard deviation sigma.
Seeds are 20120925 + the workload's number (1..5); ensemble member e uses
20120925 + 4 + 1000 + e.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20120925


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_field(shape, lengths, sigma: float, ell: float, seed: int) -> np.ndarray:
    """Stationary Gaussian field with covariance exp(-r^2/(2 ell^2)) on a
    periodic grid of ``shape`` (nz, ny, nx) covering ``lengths`` (lz, ly, lx).
    Returned flat (x fastest), rescaled to mean 0 and standard deviation sigma."""
    shape = tuple(int(s) for s in shape)
    white = rng_for(seed).standard_normal(shape)
    axes = []
    for n, L in zip(shape, lengths):
        h = L / n
        k = np.arange(n)
        dist = np.minimum(k, n - k) * h  # periodic (minimum-image) distance
        axes.append(dist)
    r2 = np.zeros(shape)
    for a, dist in enumerate(axes):
        sh = [1] * len(shape)
        sh[a] = shape[a]
        r2 = r2 + (dist**2).reshape(sh)
    cov = np.exp(-r2 / (2.0 * ell * ell))
    spec = np.real(np.fft.fftn(cov))
    spec = np.maximum(spec, 0.0)
    f = np.real(np.fft.ifftn(np.sqrt(spec) * np.fft.fftn(white)))
    f = f - f.mean()
    sd = f.std()
    f = f * (sigma / sd) if sd > 0 else f
    return f.reshape(-1)


def layered_channels(n: int, nlayers: int, nchannels: int, width: int, contrast: float,
                     seed: int) -> np.ndarray:
    """ln k on an n^3 grid: ``nlayers`` horizontal layers (z slabs) with
    ln k ~ N(0, 1) each, plus ``nchannels`` x-aligned channels of
    width x width cells at distinct, non-overlapping (y, z) blocks with
    ln k = ln(contrast).  Flat, x fastest."""
    rng = rng_for(seed)
    layer_vals = rng.standard_normal(nlayers)
    lnk = np.empty((n, n, n))
    thick = n // nlayers
    for L in range(nlayers):
        z1 = n if L == nlayers - 1 else (L + 1) * thick
        lnk[L * thick : z1, :, :] = layer_vals[L]
    blocks = n // width
    picks = rng.choice(blocks * blocks, size=nchannels, replace=False)
    for b in picks:
        bz, by = divmod(int(b), blocks)
        lnk[bz * width : (bz + 1) * width, by * width : (by + 1) * width, :] = np.log(contrast)
    return lnk.reshape(-1)


def rhoc_for_peclet(peclet: float, lam: float, velocity: float, length: float = 1.0) -> float:
    """Volumetric heat capacity (rho c) that makes Pe = (rho c) U L / lambda."""
    return peclet * lam / (velocity * length)


@dataclass
class Workload:
    """Fields and constants of one synthetic workload (flat FP64 arrays)."""

    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    lnk: np.ndarray
    phi: np.ndarray
    lam: np.ndarray
    T0: np.ndarray
    steps: int
    dt: float
    tol: float = 1e-6
    peclet: float = 50.0
    T_inflow: float = 80.0
    head_drop: float = 1.0
    fluid_model: int = 0
    velocity_scale: str = "inflow"  # "inflow": net inflow per width; "max": max face speed
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def heat2d(n: int = 64, sigma: float = 1.0, ell: float = 0.1, seed: int = SEED_BASE + 1,
           steps: int = 20, dt: float = 0.05, name: str = "heat2d_64") -> Workload:
    """2D TPFA heat transport on the unit square (the 64x64 workload and its
    resized variants used by the tests)."""
    lnk = gaussian_field((1, n, n), (1.0, 1.0, 1.0), sigma, ell, seed)
    N = n * n
    return Workload(name, 2, n, n, 1, lnk, np.full(N, 0.2), np.full(N, 2.0),
                    np.full(N, 20.0), steps, dt, 1e-6, 50.0, 80.0, 1.0, 0, "inflow")


def heat2d_rect(nx: int, ny: int, sigma: float = 1.0, ell: float = 0.1, seed: int = SEED_BASE + 1,
                steps: int = 5, dt: float = 0.05) -> Workload:
    """Rectangular-grid variant (ragged sizes for tile-edge tests)."""
    lnk = gaussian_field((1, ny, nx), (1.0, 1.0, 1.0), sigma, ell, seed)
    N = nx * ny
    return Workload(f"heat2d_{nx}x{ny}", 2, nx, ny, 1, lnk, np.full(N, 0.2), np.full(N, 2.0),
                    np.full(N, 20.0), steps, dt, 1e-6, 50.0, 80.0, 1.0, 0, "inflow")


def coupled2d(n: int = 1024, seed: int = SEED_BASE + 2, steps: int = 200, dt: float = 0.005,
              sigma: float = 2.0, ell: float = 0.02) -> Workload:
    """2D sequential pressure/temperature coupling with T-dependent fluid laws."""
    lnk = gaussian_field((1, n, n), (1.0, 1.0, 1.0), sigma, ell, seed)
    N = n * n
    return Workload(f"coupled2d_{n}", 2, n, n, 1, lnk, np.full(N, 0.2), np.full(N, 2.0),
                    np.full(N, 20.0), steps, dt, 1e-6, 50.0, 80.0, 1.0, 1, "inflow")


def channels3d(n: int = 256, seed: int = SEED_BASE + 3, steps: int = 50, dt: float | None = None,
               nchannels: int = 8, nlayers: int = 16) -> Workload:
    """3D layered reservoir with high-permeability channels (contrast 1e4).
    Velocities are scaled so that the largest face speed is 1; Pe = 1e3 with
    lambda = 1 gives (rho c) = 1e3; dt = 8 h (8 cells per step in channels)."""
    width = max(1, n // 32)
    lnk = layered_channels(n, min(nlayers, n), nchannels, width, 1e4, seed)
    N = n**3
    if dt is None:
        dt = 8.0 / n
    return Workload(f"channels3d_{n}", 3, n, n, n, lnk, np.full(N, 0.2), np.full(N, 1.0),
                    np.full(N, 20.0), steps, dt, 1e-6, 1e3, 80.0, 1.0, 0, "max")


def ensemble_sizes(members: int = 512, seed: int = SEED_BASE + 4):
    """Grid sizes n_e ~ U{64..512} and sigma_e ~ U[0.5, 2.5] of the ensemble."""
    rng = rng_for(seed)
    sizes = rng.integers(64, 513, size=members)
    sigmas = rng.uniform(0.5, 2.5, size=members)
    return sizes, sigmas


def ensemble_member(e: int, members: int = 512) -> Workload:
    sizes, sigmas = ensemble_sizes(members)
    n = int(sizes[e])
    return heat2d(n, float(sigmas[e]), 0.1, SEED_BASE + 4 + 1000 + e, 30, 0.05,
                  name=f"ensemble2d_{e}")


def adjoint3d(n: int = 128, seed: int = SEED_BASE + 5, steps: int = 60, n_obs: int = 16):
    """The adjoint workload: the layered channel reservoir of ``channels3d`` on
    n^3 cells (its own seed), 60 steps, and n_obs seeded observation cells
    with synthetic observed temperatures in [20, 80].  Returns (Workload, obs,
    data)."""
    wl = channels3d(n, seed=seed, steps=steps)
    rng = rng_for(seed + 1)
    obs = np.sort(rng.choice(wl.n, size=n_obs, replace=False))
    data = rng.uniform(20.0, 80.0, size=n_obs)
    return wl, obs, data
