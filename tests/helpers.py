"""Test helpers: direction mapping between the two numberings of a lattice and
conversions between the oracle's numpy arrays and the GPU's canonical
tensors.  No lattice Boltzmann arithmetic lives here."""
from __future__ import annotations

import numpy as np

import oracle


def perm_oracle_to(c_other: np.ndarray) -> np.ndarray:
    """p with c_other[p[k]] == c_oracle[k] (both [q, 3], q = 15, 19 or 27)."""
    c_o, _, _ = oracle.lattice(len(c_other))
    index = {tuple(int(v) for v in c): i for i, c in enumerate(c_other)}
    return np.array([index[tuple(int(v) for v in c)] for c in c_o], dtype=np.int64)


def sorted_order(c: np.ndarray) -> np.ndarray:
    """Indices of the directions of c sorted by (cx, cy, cz)."""
    keys = [tuple(int(v) for v in row) for row in c]
    return np.array(sorted(range(len(keys)), key=lambda i: keys[i]), dtype=np.int64)


def noisy_equilibrium(cfg: "oracle.Config", seed: int, amp: float = 0.02, drho: float = 0.01, umax: float = 0.04):
    """Oracle-order populations feq(rho, u) * (1 + noise): a non-equilibrium
    state built from the shared seeded generators."""
    from paper_2208_05429_gb300 import inputs
    rho, u = inputs.random_density_velocity(cfg.nx, cfg.ny, cfg.nz, seed, drho=drho, umax=umax)
    f = oracle.init_equilibrium(cfg, rho, u)
    noise = inputs.population_noise(cfg.nx, cfg.ny, cfg.nz, seed + 1, amp=amp, q=cfg.q)
    c_o, _, _ = oracle.lattice(cfg.q)
    order = sorted_order(c_o)          # noise[k] belongs to the k-th sorted vector
    f_noise = np.empty_like(noise)
    f_noise[order] = noise
    return f * (1.0 + f_noise)


def relmax(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))
