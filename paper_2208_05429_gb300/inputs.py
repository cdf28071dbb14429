"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Nothing here computes any part of the lattice Boltzmann update: these are the
initial fields, force fields, targets and sample positions of the workloads,
built from numpy random generators with fixed seeds.  Arrays use the
canonical layout [..., nz, ny, nx].

Workloads (synthetic stand-ins: the paper's only workload is a 3D
lid-driven cavity cube, Sec. 5.1, L = 64..896, Sec. 5.2):
  * cavity: fluid at rest, rho = 1 (no input arrays needed);
  * Taylor-Green: u = U0 (sin x cos y cos z, -cos x sin y cos z, 0) on the
    2 pi periodic grid x_k = 2 pi k / N;
  * differentiable channel: per-cell body force N(0, sigma^2) plus a uniform
    bias along x; loss target is a separable parabola on the outlet plane.
"""
from __future__ import annotations

import numpy as np

SEED_FORCE = 2208
SEED_CELLS = 5429


def taylor_green_velocity(nx: int, ny: int, nz: int, U0: float) -> np.ndarray:
    """u[3, nz, ny, nx] of the Taylor-Green vortex (float64)."""
    x = 2.0 * np.pi * np.arange(nx) / nx
    y = 2.0 * np.pi * np.arange(ny) / ny
    z = 2.0 * np.pi * np.arange(nz) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    u[0] = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def shear_wave_velocity(nx: int, ny: int, nz: int, U0: float, axis_u: int = 0, axis_k: int = 1,
                        mode: int = 1) -> np.ndarray:
    """u[3, ...] with u_{axis_u} = U0 sin(2 pi mode r / N) along axis_k."""
    shape = (nz, ny, nx)
    n = (nx, ny, nz)[axis_k]
    r = np.arange(n)
    prof = U0 * np.sin(2.0 * np.pi * mode * r / n)
    bshape = [1, 1, 1]
    bshape[2 - axis_k] = n
    u = np.zeros((3, *shape))
    u[axis_u] = np.broadcast_to(prof.reshape(bshape), shape)
    return u


def channel_force(nx: int, ny: int, nz: int, seed: int = SEED_FORCE, sigma: float = 1e-6,
                  bias_x: float = 1e-5) -> np.ndarray:
    """Per-cell body force F[3, nz, ny, nx] (float32): N(0, sigma^2) + bias_x along x."""
    rng = np.random.default_rng(seed)
    F = rng.normal(0.0, sigma, size=(3, nz, ny, nx))
    F[0] += bias_x
    return F.astype(np.float32)


def parabolic_target(ny: int, nz: int, Ut: float = 1e-3) -> np.ndarray:
    """Target u_x(y, z) on an outlet plane: Ut * 16 (y+1/2)(ny-y-1/2)(z+1/2)(nz-z-1/2) / (ny^2 nz^2)."""
    y = np.arange(ny) + 0.5
    z = np.arange(nz) + 0.5
    return Ut * 16.0 * np.outer(z * (nz - z), y * (ny - y)) / (ny * ny * nz * nz)


def random_density_velocity(nx: int, ny: int, nz: int, seed: int, drho: float = 0.01, umax: float = 0.05):
    """rho[nz,ny,nx] = 1 + U(-drho, drho), u[3,...] = U(-umax, umax) (float64)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rng.uniform(-drho, drho, size=(nz, ny, nx))
    u = rng.uniform(-umax, umax, size=(3, nz, ny, nx))
    return rho, u


def population_noise(nx: int, ny: int, nz: int, seed: int, amp: float = 0.02, q: int = 19) -> np.ndarray:
    """noise[q, nz, ny, nx] = U(-amp, amp); entry k belongs to the k-th
    velocity of D3Q<q> in sorted (cx, cy, cz) order, so both implementations
    can map it onto their own direction numbering."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(q, nz, ny, nx))


def sample_cells(nx: int, ny: int, nz: int, k: int, seed: int = SEED_CELLS) -> np.ndarray:
    """k distinct cells as an int64 array [k, 3] of (x, y, z)."""
    rng = np.random.default_rng(seed)
    flat = rng.choice(nx * ny * nz, size=k, replace=False)
    x = flat % nx
    y = (flat // nx) % ny
    z = flat // (nx * ny)
    return np.stack([x, y, z], axis=1).astype(np.int64)
