"""The oracle's hand-derived discrete adjoint against central finite
differences of the oracle's own forward map (FP64), on D3Q19 and on the
D3Q15 and D3Q27 lattices the same formulas serve."""
import numpy as np
import pytest

import oracle
from oracle import BC_PERIODIC, BC_WALL, BC_LID, FORCE_FIELD
from paper_2208_05429_gb300 import inputs
from helpers import noisy_equilibrium


def _channel(nx=6, ny=5, nz=4, tau=0.6, lid=False, q=19):
    bc = (BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL, BC_WALL, BC_LID if lid else BC_WALL)
    cfg = oracle.Config(nx=nx, ny=ny, nz=nz, tau=tau, bc=bc, u_lid=(0.03, 0.0, 0.0), force_mode=FORCE_FIELD, q=q)
    cfg.force_field = inputs.channel_force(nx, ny, nz, seed=2208, sigma=1e-4, bias_x=1e-4).astype(np.float64)
    return cfg


def _loss_parts(cfg, target, weights_rho):
    def loss(f):
        rho, u = oracle.moments(cfg, f)
        return float(np.sum((u[0, :, :, -1] - target) ** 2) + np.sum(weights_rho * (rho - 1.0)))

    def dLdu(rho, u):
        g = np.zeros_like(u)
        g[0, :, :, -1] = 2.0 * (u[0, :, :, -1] - target)
        return g

    def dLdrho(rho, u):
        return weights_rho

    return loss, dLdu, dLdrho


@pytest.mark.parametrize("q", [19, 15, 27])
@pytest.mark.parametrize("lid", [False, True])
def test_adjoint_matches_central_differences(lid, q):
    cfg = _channel(lid=lid, q=q)
    T = 6
    f0 = noisy_equilibrium(cfg, seed=17, amp=0.01)
    target = inputs.parabolic_target(cfg.ny, cfg.nz, Ut=1e-2)
    wr = np.random.default_rng(3).uniform(-1, 1, size=cfg.shape)
    loss, dLdu, dLdrho = _loss_parts(cfg, target, wr)
    lam0, gF = oracle.adjoint_run(cfg, f0, T, dLdu, dLdrho)

    def L_of(f_init, Ffield):
        c2 = _channel(lid=lid, q=q)
        c2.force_field = Ffield
        return loss(oracle.run(c2, f_init, T))

    rng = np.random.default_rng(5429)
    F0 = cfg.force_field.copy()
    for _ in range(8):
        a, z, y, x = rng.integers(3), rng.integers(cfg.nz), rng.integers(cfg.ny), rng.integers(cfg.nx)
        h = 1e-6
        Fp, Fm = F0.copy(), F0.copy()
        Fp[a, z, y, x] += h
        Fm[a, z, y, x] -= h
        fd = (L_of(f0, Fp) - L_of(f0, Fm)) / (2 * h)
        assert abs(gF[a, z, y, x] - fd) <= 1e-6 * max(abs(fd), 1e-3), (a, z, y, x, gF[a, z, y, x], fd)
    for _ in range(8):
        i, z, y, x = rng.integers(q), rng.integers(cfg.nz), rng.integers(cfg.ny), rng.integers(cfg.nx)
        h = 1e-6
        fp, fm = f0.copy(), f0.copy()
        fp[i, z, y, x] += h
        fm[i, z, y, x] -= h
        fd = (L_of(fp, F0) - L_of(fm, F0)) / (2 * h)
        assert abs(lam0[i, z, y, x] - fd) <= 1e-6 * max(abs(fd), 1e-3), (i, z, y, x, lam0[i, z, y, x], fd)


@pytest.mark.parametrize("q", [19, 15, 27])
def test_adjoint_step_is_transpose(q):
    """<lam, J v> = <J^T lam, v> for the one-step Jacobian J (J v by central
    differences of the step, which is quadratic-free enough for h = 1e-6)."""
    cfg = _channel(nx=5, ny=4, nz=4, lid=True, q=q)
    f = noisy_equilibrium(cfg, seed=8, amp=0.02)
    rng = np.random.default_rng(9)
    lam = rng.normal(size=f.shape)
    v = rng.normal(size=f.shape)
    h = 1e-6
    Jv = (oracle.step(cfg, f + h * v) - oracle.step(cfg, f - h * v)) / (2 * h)
    gF = np.zeros((3, *cfg.shape))
    JTlam = oracle.adjoint_step(cfg, f, lam, gF)
    lhs, rhs = np.sum(lam * Jv), np.sum(JTlam * v)
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)
