"""Absolute pins of the oracle's global sums (mass, momentum, kinetic energy).

The sums are defined on the moments of each cell: M = sum rho, P = sum of the
first moment sum_i f_i c_i (no half force), KE = sum 1/2 rho |u|^2 with
u = (sum_i f_i c_i + F/2) / rho.  An equilibrium feq(rho, u) reproduces rho
and rho u exactly (second-order Hermite equilibrium), so on states built from
known density and velocity fields every expected value below comes from
those input fields alone, never from the oracle.  A dropped rest
population, a missing 1/2 in KE, the half force left out of u or put into
P, or a sign slip in a velocity component each fail one of these tests.
"""
import numpy as np
import pytest

import oracle
from oracle import FORCE_FIELD, FORCE_UNIFORM
from paper_2208_05429_gb300 import inputs


def _uniform_state(cfg, rho0, u0):
    rho = np.full(cfg.shape, rho0)
    u = np.zeros((3, *cfg.shape))
    for a in range(3):
        u[a] = u0[a]
    return oracle.init_equilibrium(cfg, rho, u)


@pytest.mark.parametrize("rho0,u0", [(1.0, (0.0, 0.0, 0.0)), (1.07, (0.04, -0.025, 0.013)),
                                     (0.93, (-0.05, 0.0, 0.031))])
def test_reduce_uniform_state(rho0, u0):
    """Periodic box at a uniform equilibrium (rho0, u0), no force:
    M = N rho0, P = N rho0 u0, KE = N rho0 |u0|^2 / 2."""
    cfg = oracle.Config(nx=7, ny=5, nz=6, tau=0.7)
    f = _uniform_state(cfg, rho0, u0)
    out = oracle.reduce(cfg, f)
    n = cfg.n
    u0 = np.array(u0)
    assert abs(out[0] - n * rho0) <= 1e-13 * n * rho0
    assert np.allclose(out[1:4], n * rho0 * u0, rtol=1e-12, atol=1e-14 * n)
    ke = 0.5 * n * rho0 * float(u0 @ u0)
    assert abs(out[4] - ke) <= 1e-12 * max(ke, 1e-300) + 1e-18


def test_reduce_uniform_state_with_force():
    """With a uniform force F the velocity carries the half force,
    u = u0 + F / (2 rho0), while P stays the bare first moment N rho0 u0."""
    F = np.array([2e-3, -1e-3, 5e-4])
    cfg = oracle.Config(nx=5, ny=6, nz=4, tau=0.8, force_mode=FORCE_UNIFORM, force_uniform=tuple(F))
    rho0, u0 = 1.04, np.array([0.03, 0.01, -0.02])
    out = oracle.reduce(cfg, _uniform_state(cfg, rho0, u0))
    n = cfg.n
    assert abs(out[0] - n * rho0) <= 1e-13 * n * rho0
    assert np.allclose(out[1:4], n * rho0 * u0, rtol=1e-12, atol=1e-14 * n)
    uf = u0 + F / (2.0 * rho0)
    ke = 0.5 * n * rho0 * float(uf @ uf)
    assert abs(out[4] - ke) <= 1e-12 * ke


def test_reduce_nonuniform_fields():
    """Equilibria of seeded non-uniform rho and u fields: the three sums are
    the sums of the input fields, and a per-cell force field enters KE only
    through u = u_in + F / (2 rho)."""
    cfg = oracle.Config(nx=9, ny=7, nz=5, tau=0.6, force_mode=FORCE_FIELD)
    Ff = inputs.channel_force(9, 7, 5, seed=31, sigma=2e-3).astype(np.float64)
    cfg.force_field = Ff
    rho, u = inputs.random_density_velocity(9, 7, 5, seed=29, drho=0.05, umax=0.05)
    f = oracle.init_equilibrium(cfg, rho, u)
    out = oracle.reduce(cfg, f)
    M = rho.sum()
    P = (rho[None] * u).reshape(3, -1).sum(axis=1)
    uf = u + Ff / (2.0 * rho[None])
    KE = float((0.5 * rho * (uf ** 2).sum(axis=0)).sum())
    assert abs(out[0] - M) <= 1e-13 * M
    assert np.allclose(out[1:4], P, rtol=1e-11, atol=1e-14)
    assert abs(out[4] - KE) <= 1e-11 * KE


def test_reduce_matches_direct_population_sums():
    """On an arbitrary (non-equilibrium) state M and P are plain sums of the
    populations weighted by 1 and c_i; the rest population is included."""
    cfg = oracle.Config(nx=6, ny=4, nz=3, tau=0.7)
    rng = np.random.default_rng(12)
    f = 0.02 + rng.random((19, *cfg.shape)) * 0.1
    c, _, _ = oracle.lattice()
    out = oracle.reduce(cfg, f)
    assert abs(out[0] - f.sum()) <= 1e-13 * f.sum()
    P = np.einsum("qa,qzyx->a", c.astype(np.float64), f)
    assert np.allclose(out[1:4], P, rtol=1e-12, atol=1e-14 * cfg.n)
    # dropping the rest population would change the mass by this much
    assert f[0].sum() > 1e3 * 1e-13 * f.sum()
