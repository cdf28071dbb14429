"""Pins of the oracle's two-relaxation-time (TRT) collision.

Closed forms and special cases that fix it without referring to the
oracle's own formula:
  * with omega- = omega+ (Lambda = (tau - 1/2)^2) TRT is BGK, cell by cell;
  * the collision conserves mass, and momentum up to the Guo source (the
    first moment of the post-collision populations is j + F);
  * half-way bounce-back with Lambda = 3/16 places the walls of a body-force
    driven channel exactly half-way for every tau: the plane Poiseuille
    profile u = F/(2 nu) (y + 1/2)(H - y - 1/2), nu = (tau - 1/2)/3, to
    rounding (the known "magic" value of the TRT wall closure);
  * a shear wave decays with nu = (tau - 1/2)/3, whatever Lambda.
A dropped 1/2 in the part split, omega- taken as omega+, or the force parts
swapped fails one of these."""
import numpy as np
import pytest

import oracle
from oracle import BC_PERIODIC, BC_WALL, COLL_TRT, FORCE_UNIFORM
from paper_2208_05429_gb300 import inputs


def _noisy_cell(seed):
    rng = np.random.default_rng(seed)
    rho, u = 1.0 + rng.uniform(-0.02, 0.02), rng.uniform(-0.05, 0.05, 3)
    f = oracle.equilibrium(rho, u)
    return f * (1.0 + rng.uniform(-0.05, 0.05, f.shape))


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.7])
def test_trt_is_bgk_when_rates_match(tau):
    lam = (tau - 0.5) ** 2
    F = np.array([1e-4, -2e-4, 5e-5])
    for seed in range(5):
        f = _noisy_cell(seed)
        assert np.allclose(oracle.collide_cell_trt(tau, lam, f, F), oracle.collide_cell(tau, f, F),
                           rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("lam", [0.02, 3.0 / 16.0, 0.7])
def test_trt_conserves_mass_and_momentum(lam):
    c, _, _ = oracle.lattice()
    F = np.array([3e-4, -1e-4, 2e-4])
    for seed in range(5):
        f = _noisy_cell(seed + 10)
        fs = oracle.collide_cell_trt(0.7, lam, f, F)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.allclose(c.T @ fs, c.T @ f + F, atol=1e-15)
        # and it is not BGK: the antisymmetric part relaxes at another rate
        assert np.max(np.abs(fs - oracle.collide_cell(0.7, f, F))) > 1e-9 or abs(lam - 0.04) < 1e-12


def _channel(tau, H, F, steps, lam):
    cfg = oracle.Config(nx=1, ny=H, nz=1, tau=tau, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL,
                                                       BC_PERIODIC, BC_PERIODIC),
                        force_mode=FORCE_UNIFORM, force_uniform=(F, 0.0, 0.0), collision=COLL_TRT, trt_lambda=lam)
    f = oracle.run(cfg, oracle.init_equilibrium(cfg), steps)
    rho, u = oracle.moments(cfg, f)
    return rho[0, :, 0], u[0, 0, :, 0]


@pytest.mark.parametrize("tau", [0.6, 0.9, 1.5])
def test_trt_poiseuille_exact_at_magic_lambda(tau):
    H, F = 8, 1e-5
    nu = (tau - 0.5) / 3.0
    steps = int(60 * H * H / nu / 3.0) + 1000
    rho, ux = _channel(tau, H, F, steps, 3.0 / 16.0)
    y = np.arange(H)
    exact = F / (2.0 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.max(np.abs(ux - exact)) / np.max(exact) < 1e-9
    # away from the magic value the wall moves (the profile slips)
    _, ux2 = _channel(tau, H, F, steps, 0.02)
    assert np.max(np.abs(ux2 - exact)) / np.max(exact) > 1e-4


def _nu_ratio(n, tau, lam):
    cfg = oracle.Config(nx=1, ny=n, nz=1, tau=tau, collision=COLL_TRT, trt_lambda=lam)
    u0 = inputs.shear_wave_velocity(1, n, 1, 1e-4, axis_u=0, axis_k=1)
    f = oracle.init_equilibrium(cfg, None, u0)
    f = oracle.run(cfg, f, 60)
    a0 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    f = oracle.run(cfg, f, 200)
    a1 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    return -np.log(a1 / a0) / ((2.0 * np.pi / n) ** 2 * 200) / ((tau - 0.5) / 3.0) - 1.0


@pytest.mark.parametrize("lam", [0.05, 3.0 / 16.0, 0.5])
def test_trt_shear_wave_viscosity(lam):
    """The decay rate of a shear wave gives nu = (tau - 1/2)/3 up to an
    O(k^2) term whose size depends on Lambda: halving k divides the
    deviation by four."""
    d32, d64 = _nu_ratio(32, 0.8, lam), _nu_ratio(64, 0.8, lam)
    assert abs(d64) < 3e-3
    assert abs(d32 / d64 - 4.0) < 0.2
