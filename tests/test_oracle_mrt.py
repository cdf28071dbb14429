"""Pins of the oracle's multiple-relaxation-time (MRT) collision in Hermite
moments: the non-equilibrium moments of order up to two relax with
omega = 1/tau, those of order three with s3 and of order four with s4.

Closed forms and special cases that fix it without referring to the
oracle's own formula:
  * s3 = s4 = omega is BGK, s3 = s4 = 1 the regularised collision, and
    (without a force) s3 = omega-, s4 = omega the TRT collision;
  * a non-equilibrium mode orthogonal (in sum_i w_i a_i b_i) to every
    polynomial of order up to three -- built here with numpy, not from the
    oracle's basis -- is multiplied by 1 - s4; an odd one orthogonal to the
    first-order polynomials by 1 - s3;
  * mass, momentum (+ F) and the stress are those of BGK;
  * a shear wave decays with nu = (tau - 1/2)/3.
A moment put in the wrong order, a rate swapped, or a basis left
non-orthogonal fails one of these."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import COLL_MRT
from paper_2208_05429_gb300 import inputs


def _cell(seed):
    rng = np.random.default_rng(seed)
    rho, u = 1.0 + rng.uniform(-0.02, 0.02), rng.uniform(-0.05, 0.05, 3)
    feq = oracle.equilibrium(rho, u)
    return rng, feq, feq * (1.0 + rng.uniform(-0.05, 0.05, feq.shape))


def _polys(order_max):
    """Monomials x^a y^b z^c of total order <= order_max, on the velocities."""
    c, _, _ = oracle.lattice()
    x, y, z = c.T.astype(np.float64)
    rows = [x ** a * y ** b * z ** e for a, b, e in itertools.product(range(5), repeat=3) if a + b + e <= order_max]
    return np.array(rows)


def _mode(rng, order_max, odd=False):
    """A population h_i = w_i phi_i whose phi is orthogonal, in the weighted
    product, to all polynomials of order <= order_max (odd: phi odd in c)."""
    c, w, opp = oracle.lattice()
    phi = rng.normal(size=len(w))
    if odd:
        phi = 0.5 * (phi - phi[opp])
    P = _polys(order_max)
    G = (P * w) @ P.T
    coef = np.linalg.lstsq(G, (P * w) @ phi, rcond=None)[0]
    phi = phi - P.T @ coef
    assert np.max(np.abs((P * w) @ phi)) < 1e-12
    return w * phi


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.7])
def test_mrt_limits(tau):
    F = np.array([1e-4, -2e-4, 5e-5])
    om = 1.0 / tau
    for seed in range(4):
        _, _, f = _cell(seed)
        assert np.allclose(oracle.collide_cell_mrt(tau, om, om, f, F), oracle.collide_cell(tau, f, F),
                           rtol=1e-13, atol=1e-16)
        assert np.allclose(oracle.collide_cell_mrt(tau, 1.0, 1.0, f, F), oracle.collide_cell_reg(tau, f, F),
                           rtol=1e-13, atol=1e-16)
        for om_m in (0.6, 1.3):
            lam = (tau - 0.5) * (1.0 / om_m - 0.5)
            assert np.allclose(oracle.collide_cell_mrt(tau, om_m, om, f), oracle.collide_cell_trt(tau, lam, f),
                               rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("s3,s4", [(1.1, 1.6), (0.7, 1.9), (1.5, 0.9)])
def test_mrt_relaxes_each_order_with_its_rate(s3, s4):
    tau = 0.7
    for seed in range(4):
        rng, feq, _ = _cell(seed + 10)
        h4 = 1e-3 * _mode(rng, 3)
        assert np.allclose(oracle.collide_cell_mrt(tau, s3, s4, feq + h4) - feq, (1.0 - s4) * h4,
                           rtol=0, atol=1e-15)
        h3 = 1e-3 * _mode(rng, 1, odd=True)
        assert np.allclose(oracle.collide_cell_mrt(tau, s3, s4, feq + h3) - feq, (1.0 - s3) * h3,
                           rtol=0, atol=1e-15)


def test_mrt_conservation_and_stress():
    c, _, _ = oracle.lattice()
    F = np.array([3e-4, -1e-4, 2e-4])
    for seed in range(5):
        _, _, f = _cell(seed + 30)
        fs = oracle.collide_cell_mrt(0.7, 1.2, 1.7, f, F)
        bgk = oracle.collide_cell(0.7, f, F)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.allclose(c.T @ fs, c.T @ f + F, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", fs, c, c), np.einsum("i,ia,ib->ab", bgk, c, c), atol=1e-15)
        assert np.max(np.abs(fs - bgk)) > 1e-7


def _nu_ratio(n, tau):
    cfg = oracle.Config(nx=1, ny=n, nz=1, tau=tau, collision=COLL_MRT, mrt_s3=1.2, mrt_s4=1.5)
    u0 = inputs.shear_wave_velocity(1, n, 1, 1e-4, axis_u=0, axis_k=1)
    f = oracle.init_equilibrium(cfg, None, u0)
    f = oracle.run(cfg, f, 60)
    a0 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    f = oracle.run(cfg, f, 200)
    a1 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
    return -np.log(a1 / a0) / ((2.0 * np.pi / n) ** 2 * 200) / ((tau - 0.5) / 3.0) - 1.0


def test_mrt_shear_wave_viscosity():
    d32, d64 = _nu_ratio(32, 0.8), _nu_ratio(64, 0.8)
    assert abs(d64) < 3e-3
    assert abs(d32 / d64 - 4.0) < 0.3
