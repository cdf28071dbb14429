"""Pins of the oracle's streaming, boundaries and forcing against conservation
laws and closed-form flows (no value here comes from the oracle itself)."""
import numpy as np
import pytest

import oracle
from oracle import BC_LID, BC_PERIODIC, BC_WALL, FORCE_FIELD, FORCE_UNIFORM
from paper_2208_05429_gb300 import inputs


def test_uniform_equilibrium_is_fixed_point():
    cfg = oracle.Config(nx=6, ny=5, nz=4, tau=0.7)
    rho = np.full(cfg.shape, 1.03)
    u = np.zeros((3, *cfg.shape))
    u[0], u[1], u[2] = 0.04, -0.02, 0.01
    f0 = oracle.init_equilibrium(cfg, rho, u)
    f = oracle.run(cfg, f0, 50)
    assert np.max(np.abs(f - f0)) < 1e-15


def test_cavity_conserves_mass_exactly():
    """Half-way bounce-back with the lid taking precedence at lid edges and
    rho_w = 1 keeps sum f constant to rounding."""
    cfg = oracle.cavity(16, 0.6)
    f0 = oracle.init_equilibrium(cfg)
    f = oracle.run(cfg, f0, 100)
    m0, m1 = f0.sum(), f.sum()
    assert abs(m1 - m0) / m0 < 1e-13
    # and the lid actually drives the flow
    _, u = oracle.moments(cfg, f)
    assert np.max(np.abs(u[0])) > 1e-3


def test_mass_conservation_other_walls():
    cfg = oracle.Config(nx=7, ny=6, nz=5, tau=0.55, bc=(BC_LID, BC_LID, BC_WALL, BC_WALL, BC_PERIODIC, BC_PERIODIC),
                        u_lid=(0.0, 0.03, 0.02))
    f0 = oracle.init_equilibrium(cfg)
    f = oracle.run(cfg, f0, 60)
    assert abs(f.sum() - f0.sum()) / f0.sum() < 1e-13


def test_periodic_force_momentum_gain():
    """In a fully periodic box every step adds exactly F to each cell's momentum."""
    cfg = oracle.Config(nx=5, ny=4, nz=3, tau=0.9, force_mode=FORCE_UNIFORM, force_uniform=(1e-4, -2e-5, 3e-5))
    rho, u = inputs.random_density_velocity(cfg.nx, cfg.ny, cfg.nz, seed=3)
    f0 = oracle.init_equilibrium(cfg, rho, u)
    P0 = oracle.reduce(cfg, f0)[1:4]
    n = 40
    P1 = oracle.reduce(cfg, oracle.run(cfg, f0, n))[1:4]
    gain = n * cfg.n * np.array(cfg.force_uniform)
    assert np.allclose(P1 - P0, gain, rtol=1e-10, atol=1e-15)


def test_force_field_momentum_gain():
    cfg = oracle.Config(nx=4, ny=4, nz=4, tau=0.7, force_mode=FORCE_FIELD)
    cfg.force_field = inputs.channel_force(4, 4, 4, seed=11, sigma=1e-4).astype(np.float64)
    f0 = oracle.init_equilibrium(cfg)
    P0 = oracle.reduce(cfg, f0)[1:4]
    P1 = oracle.reduce(cfg, oracle.run(cfg, f0, 10))[1:4]
    assert np.allclose(P1 - P0, 10 * cfg.force_field.reshape(3, -1).sum(axis=1), rtol=1e-10, atol=1e-15)


def test_couette_profile_exact():
    """Wall at z = -1/2, lid at z = nz - 1/2 moving with U: the steady profile
    is u_x = U (z + 1/2) / nz at every cell (pins the lid term's sign and size)."""
    U, nz = 0.02, 8
    cfg = oracle.Config(nx=1, ny=1, nz=nz, tau=0.8, bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_LID),
                        u_lid=(U, 0.0, 0.0))
    f = oracle.run(cfg, oracle.init_equilibrium(cfg), 4000)
    rho, u = oracle.moments(cfg, f)
    z = np.arange(nz) + 0.5
    assert np.allclose(u[0, :, 0, 0], U * z / nz, rtol=0, atol=1e-12 * U)
    assert np.allclose(u[1:], 0.0, atol=1e-13)


def _poiseuille(tau, H, F, steps):
    cfg = oracle.Config(nx=1, ny=H, nz=1, tau=tau, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL, BC_PERIODIC, BC_PERIODIC),
                        force_mode=FORCE_UNIFORM, force_uniform=(F, 0.0, 0.0))
    f = oracle.run(cfg, oracle.init_equilibrium(cfg), steps)
    rho, u = oracle.moments(cfg, f)
    return rho[0, :, 0], u[0, 0, :, 0]


def test_poiseuille_exact_at_magic_tau():
    """With (tau - 1/2)^2 = 3/16 half-way bounce-back puts the walls exactly
    at y = -1/2 and H - 1/2: u = F/(2 nu) (y + 1/2)(H - y - 1/2), nu = (tau - 1/2)/3."""
    tau = 0.5 + np.sqrt(3.0) / 4.0
    H, F = 8, 1e-5
    rho, ux = _poiseuille(tau, H, F, 3000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = F / (2.0 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.max(np.abs(ux - exact)) / np.max(exact) < 1e-10
    assert np.allclose(rho, 1.0, atol=1e-14)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_poiseuille_curvature_any_tau(tau):
    """Away from the magic tau the bulk profile is still the exact parabola
    of curvature -F/nu (only a uniform slip differs)."""
    H, F = 10, 1e-5
    nu = (tau - 0.5) / 3.0
    steps = int(40 * H * H / nu / 3.0) + 500
    rho, ux = _poiseuille(tau, H, F, steps)
    curv = ux[2:] - 2.0 * ux[1:-1] + ux[:-2]
    assert np.allclose(curv, -F / nu, rtol=1e-8)
    assert np.allclose(ux, ux[::-1], rtol=1e-12)


def _decay_rate(tau, n, steps=(60, 260)):
    cfg = oracle.Config(nx=1, ny=n, nz=1, tau=tau)
    u0 = inputs.shear_wave_velocity(1, n, 1, 1e-4, axis_u=0, axis_k=1)
    f = oracle.init_equilibrium(cfg, None, u0)
    f = oracle.run(cfg, f, steps[0])
    a0 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    f = oracle.run(cfg, f, steps[1] - steps[0])
    a1 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    k2 = (2.0 * np.pi / n) ** 2
    return -np.log(a1 / a0) / (k2 * (steps[1] - steps[0]))


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_shear_wave_viscosity(tau):
    """A shear wave decays with the kinematic viscosity nu = (tau - 1/2)/3, up
    to an O(k^2) lattice error that shrinks fourfold when the grid doubles."""
    nu = (tau - 0.5) / 3.0
    e32 = abs(_decay_rate(tau, 32) / nu - 1.0)
    e64 = abs(_decay_rate(tau, 64, steps=(240, 1040)) / nu - 1.0)
    assert e32 < 1e-2
    assert e64 < 0.35 * e32 + 1e-6


def test_taylor_green_energy_decay():
    """3D Taylor-Green vortex, small amplitude: KE ~ exp(-2 nu |k|^2 t), |k|^2 = 3 (2 pi / N)^2."""
    n, tau = 16, 0.8
    nu = (tau - 0.5) / 3.0
    cfg = oracle.Config(nx=n, ny=n, nz=n, tau=tau)
    u0 = inputs.taylor_green_velocity(n, n, n, 1e-4)
    f = oracle.run(cfg, oracle.init_equilibrium(cfg, None, u0), 20)
    ke0 = oracle.reduce(cfg, f)[4]
    t = 60
    ke1 = oracle.reduce(cfg, oracle.run(cfg, f, t))[4]
    k2 = 3.0 * (2.0 * np.pi / n) ** 2
    rate = -np.log(ke1 / ke0) / (2.0 * k2 * t)
    assert abs(rate / nu - 1.0) < 3e-2


def test_step_cells_matches_step():
    """Sampled single-cell stepping equals the full step (bit for bit)."""
    from helpers import noisy_equilibrium
    cfg = oracle.cavity(9, 0.62, u_lid=(0.05, 0.01, 0.0), ny=7, nz=6)
    cfg.force_mode = FORCE_UNIFORM
    cfg.force_uniform = (1e-5, 0.0, -2e-6)
    f = noisy_equilibrium(cfg, seed=21)
    full = oracle.step(cfg, f)
    cells = inputs.sample_cells(cfg.nx, cfg.ny, cfg.nz, 60, seed=4)
    got = oracle.step_cells(cfg, f, cells)
    exp = np.stack([full[:, z, y, x] for x, y, z in cells])
    assert np.array_equal(got, exp)
