"""Pins of the oracle's regularised BGK collision.

Closed forms and special cases that fix it without referring to the
oracle's own formula:
  * a non-equilibrium part that already lies in the second-order Hermite
    space (w_i (9/2) Q_i : A, any symmetric A) is kept whole, so the
    collision equals BGK there;
  * with a body force f - feq carries momentum -F/2, which the projection
    keeps (its first-order part): without it the momentum gain would not be
    F;
  * a non-equilibrium part without mass, momentum or stress (a "ghost"
    mode) is removed entirely: the post-collision state is feq, where BGK
    keeps (1 - omega) of it;
  * on any state the collision conserves mass, gains momentum F (Guo), and
    leaves the same stress as BGK (the projection keeps Pi exactly, by the
    fourth-order isotropy of D3Q19);
  * a shear wave decays with nu = (tau - 1/2)/3.
A dropped 1/3 in Q_i, a wrong 9/2, or the non-equilibrium taken from f
instead of f - feq fails one of these."""
import numpy as np
import pytest

import oracle
from oracle import COLL_REG
from paper_2208_05429_gb300 import inputs


def _cell_state(seed):
    rng = np.random.default_rng(seed)
    rho, u = 1.0 + rng.uniform(-0.02, 0.02), rng.uniform(-0.05, 0.05, 3)
    return rng, rho, u, oracle.equilibrium(rho, u)


def _hermite2(A):
    c, w, _ = oracle.lattice()
    cc = np.einsum("ia,ab,ib->i", c, A, c)
    return w * 4.5 * (cc - np.trace(A) / 3.0)


def _moment_matrix():
    """Rows: 1, c_a (3), c_a c_b (6) -- the moments a ghost mode lacks."""
    c, _, _ = oracle.lattice()
    rows = [np.ones(len(c))] + [c[:, a] for a in range(3)]
    rows += [c[:, a] * c[:, b] for a in range(3) for b in range(a, 3)]
    return np.array(rows, dtype=np.float64)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.7])
def test_reg_is_bgk_on_second_order_non_equilibrium(tau):
    for seed in range(5):
        rng, rho, u, feq = _cell_state(seed)
        A = rng.normal(size=(3, 3)) * 1e-3
        f = feq + _hermite2(A + A.T)
        assert np.allclose(oracle.collide_cell_reg(tau, f), oracle.collide_cell(tau, f), rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.7])
def test_reg_removes_ghost_modes(tau):
    M = _moment_matrix()
    for seed in range(5):
        rng, rho, u, feq = _cell_state(seed + 20)
        r = rng.normal(size=feq.shape)
        h = r - M.T @ np.linalg.solve(M @ M.T, M @ r)
        assert np.max(np.abs(M @ h)) < 1e-12
        f = feq + 1e-3 * h
        assert np.allclose(oracle.collide_cell_reg(tau, f), feq, rtol=0, atol=1e-15)
        # BGK keeps (1 - omega) of the ghost
        bgk = oracle.collide_cell(tau, f)
        assert np.allclose(bgk - feq, (1.0 - 1.0 / tau) * 1e-3 * h, rtol=1e-9, atol=1e-17)


def test_reg_conservation_and_stress():
    c, _, _ = oracle.lattice()
    F = np.array([3e-4, -1e-4, 2e-4])
    for seed in range(5):
        rng, rho, u, feq = _cell_state(seed + 40)
        f = feq * (1.0 + rng.uniform(-0.05, 0.05, feq.shape))
        fs = oracle.collide_cell_reg(0.7, f, F)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.allclose(c.T @ fs, c.T @ f + F, atol=1e-15)
        bgk = oracle.collide_cell(0.7, f, F)
        pi_reg = np.einsum("i,ia,ib->ab", fs, c, c)
        pi_bgk = np.einsum("i,ia,ib->ab", bgk, c, c)
        assert np.allclose(pi_reg, pi_bgk, rtol=0, atol=1e-15)
        # and it is not BGK: the random noise has ghost parts
        assert np.max(np.abs(fs - bgk)) > 1e-6


def _nu_ratio(n, tau):
    cfg = oracle.Config(nx=1, ny=n, nz=1, tau=tau, collision=COLL_REG)
    u0 = inputs.shear_wave_velocity(1, n, 1, 1e-4, axis_u=0, axis_k=1)
    f = oracle.init_equilibrium(cfg, None, u0)
    f = oracle.run(cfg, f, 60)
    a0 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    f = oracle.run(cfg, f, 200)
    a1 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    return -np.log(a1 / a0) / ((2.0 * np.pi / n) ** 2 * 200) / ((tau - 0.5) / 3.0) - 1.0


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_reg_shear_wave_viscosity(tau):
    """nu = (tau - 1/2)/3 up to an O(k^2) term: halving k divides the
    deviation by about four."""
    d32, d64 = _nu_ratio(32, tau), _nu_ratio(64, tau)
    assert abs(d64) < 3e-3
    assert abs(d32 / d64 - 4.0) < 0.3
