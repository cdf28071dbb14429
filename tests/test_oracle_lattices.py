"""Pins of the oracle's D3Q15 and D3Q27 lattices (the other two cubic velocity
sets for which the paper's dependency guard holds, Sec. 4.1) without referring
to the oracle's own formulas:
  * the vector sets and their half-neighbour order (directions 1..H have -1
    as first non-zero component, i + H is the opposite of i, Sec. 3);
  * the weights through the moment identities up to fourth order, which fix
    them uniquely on each set;
  * equilibrium moments, collision invariants and the special cases of the
    TRT and regularised forms;
  * the separately written numpy brute force on tiny grids (walls, lids,
    uniform and per-cell force);
  * closed-form flows: rest state, mass conservation, momentum gain,
    Couette, Poiseuille, shear-wave viscosity nu = (tau - 1/2)/3.
A transposed table entry, a wrong weight class, a dropped term or a wrong
opposite fails one of them."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import BC_LID, BC_PERIODIC, BC_WALL, COLL_REG, COLL_TRT, FORCE_FIELD, FORCE_UNIFORM, brute
from paper_2208_05429_gb300 import inputs
from helpers import noisy_equilibrium

QS = (15, 27)
# squared lengths of the vectors each lattice holds
NORMS = {15: {0, 1, 3}, 19: {0, 1, 2}, 27: {0, 1, 2, 3}}


@pytest.mark.parametrize("q", QS + (19,))
def test_vector_set_and_half_neighbour_order(q):
    c, w, opp = oracle.lattice(q)
    vecs = [tuple(int(a) for a in v) for v in c]
    expected = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) in NORMS[q]}
    assert len(vecs) == q and set(vecs) == expected
    h = (q - 1) // 2
    assert vecs[0] == (0, 0, 0) and opp[0] == 0
    for i in range(1, h + 1):
        assert next(a for a in vecs[i] if a != 0) == -1
        assert np.array_equal(c[i + h], -c[i])
        assert opp[i] == i + h and opp[i + h] == i
    # one weight per squared length
    for i in range(q):
        for j in range(q):
            if (c[i] ** 2).sum() == (c[j] ** 2).sum():
                assert w[i] == w[j]


@pytest.mark.parametrize("q", QS + (19,))
def test_weights_from_moment_identities(q):
    """sum w = 1, sum w c c = I/3, sum w c^4 = 3 delta/9 (fourth-order isotropy):
    on D3Q15 and D3Q19 these fix the weights of the squared-length classes; on
    D3Q27, the tensor product of three D1Q3 sets, the product rule
    sum w cx^2 cy^2 cz^2 = (1/3)^3 fixes the last one."""
    c, w, _ = oracle.lattice(q)
    cf = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("q,qa->a", w, cf), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, cf, cf), np.eye(3) / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, cf, cf, cf), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, cf, cf, cf, cf), iso4, atol=1e-16)
    # and the class weights solve those identities uniquely: least squares
    # on the identities' rows gives back the table
    norms = sorted(NORMS[q])
    cls = [np.where((c ** 2).sum(axis=1) == n)[0] for n in norms]
    rows, rhs = [], []
    rows.append([len(k) for k in cls]); rhs.append(1.0)                                  # sum w
    rows.append([float((cf[k, 0] ** 2).sum()) for k in cls]); rhs.append(1.0 / 3.0)      # sum w cx^2
    rows.append([float((cf[k, 0] ** 4).sum()) for k in cls]); rhs.append(1.0 / 3.0)      # sum w cx^4
    rows.append([float((cf[k, 0] ** 2 * cf[k, 1] ** 2).sum()) for k in cls]); rhs.append(1.0 / 9.0)
    if q == 27:
        rows.append([float((cf[k, 0] ** 2 * cf[k, 1] ** 2 * cf[k, 2] ** 2).sum()) for k in cls]); rhs.append(1.0 / 27.0)
    sol, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    assert np.linalg.matrix_rank(np.array(rows)) == len(norms)
    for k, wk in zip(cls, sol):
        assert np.allclose(w[k], wk, rtol=1e-14)


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("seed", range(3))
def test_equilibrium_moments(q, seed):
    rng = np.random.default_rng(seed)
    rho, u = 1.0 + rng.uniform(-0.2, 0.2), rng.uniform(-0.1, 0.1, size=3)
    feq = oracle.equilibrium(rho, u, q)
    c, _, _ = oracle.lattice(q)
    cf = c.astype(np.float64)
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(cf.T @ feq, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("q,qa,qb->ab", feq, cf, cf), rho * np.outer(u, u) + rho / 3.0 * np.eye(3),
                       atol=1e-15)


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("seed", range(3))
def test_collision_invariants(q, seed):
    """Every collision keeps mass and adds exactly F to the momentum; BGK
    relaxes f - feq by 1 - omega; feq is a fixed point."""
    rng = np.random.default_rng(100 + seed)
    c, w, _ = oracle.lattice(q)
    cf = c.astype(np.float64)
    tau = rng.uniform(0.51, 2.0)
    f = w * (1.0 + rng.uniform(-0.3, 0.3, size=q))
    F = rng.uniform(-1e-3, 1e-3, size=3)
    for coll in (oracle.COLL_BGK, COLL_TRT, COLL_REG):
        fs = oracle.collide_cell_q(q, tau, f, F, collision=coll)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.allclose(cf.T @ fs, cf.T @ f + F, atol=1e-16)
    rho = f.sum()
    feq = oracle.equilibrium(rho, (cf.T @ f) / rho, q)
    assert np.allclose(oracle.collide_cell_q(q, tau, f) - feq, (1.0 - 1.0 / tau) * (f - feq), atol=1e-16)
    for coll in (oracle.COLL_BGK, COLL_TRT, COLL_REG):
        assert np.allclose(oracle.collide_cell_q(q, tau, feq, collision=coll), feq, atol=1e-16)


@pytest.mark.parametrize("q", QS)
def test_trt_and_regularised_special_cases(q):
    """TRT with omega- = omega+ (Lambda = (tau - 1/2)^2) is BGK; the
    regularised form equals BGK on a state whose non-equilibrium part is of
    Hermite order <= 2 and removes a mode orthogonal to those polynomials."""
    rng = np.random.default_rng(7)
    c, w, _ = oracle.lattice(q)
    cf = c.astype(np.float64)
    tau = 0.8
    F = np.array([2e-4, -1e-4, 5e-5])
    f = w * (1.0 + rng.uniform(-0.2, 0.2, size=q))
    lam = (tau - 0.5) ** 2
    assert np.allclose(oracle.collide_cell_q(q, tau, f, F, collision=COLL_TRT, lam=lam),
                       oracle.collide_cell_q(q, tau, f, F), rtol=1e-13, atol=1e-16)
    rho, u = 1.01, np.array([0.03, -0.02, 0.01])
    feq = oracle.equilibrium(rho, u, q)
    J = np.zeros(3)          # keep the momentum: J = 0 (F = 0 below)
    Pi = rng.normal(size=(3, 3)) * 1e-3
    Pi = 0.5 * (Pi + Pi.T)
    # second-order Hermite part with zero mass: sum_i w_i Q_i:Pi = 0 holds for any Pi
    Qi = np.einsum("qa,qb->qab", cf, cf) - np.eye(3) / 3.0
    f2 = feq + w * (3.0 * cf @ J + 4.5 * np.einsum("qab,ab->q", Qi, Pi))
    assert np.allclose(oracle.collide_cell_q(q, tau, f2, collision=COLL_REG), oracle.collide_cell_q(q, tau, f2),
                       rtol=0, atol=1e-16)
    # a ghost mode: phi orthogonal (weight w) to all polynomials of order <= 2
    P = np.array([cf[:, 0] ** a * cf[:, 1] ** b * cf[:, 2] ** e
                  for a, b, e in itertools.product(range(3), repeat=3) if a + b + e <= 2])
    phi = rng.normal(size=q)
    coef = np.linalg.lstsq((P * w) @ P.T, (P * w) @ phi, rcond=None)[0]
    phi -= P.T @ coef
    assert np.max(np.abs((P * w) @ phi)) < 1e-12
    g = feq + 1e-3 * w * phi
    assert np.allclose(oracle.collide_cell_q(q, tau, g, collision=COLL_REG), feq, rtol=0, atol=1e-16)


def _to_brute(f_oracle, q):
    c_o, _, _ = oracle.lattice(q)
    c_b, _ = brute.velocity_set(q)
    idx = {tuple(v): k for k, v in enumerate(c_o)}
    return np.stack([f_oracle[idx[tuple(v)]] for v in c_b])


BRUTE_CASES = {
    "cavity": dict(nx=8, ny=8, nz=8, tau=0.6, bc=(BC_WALL,) * 5 + (BC_LID,), u_lid=(0.05, 0.0, 0.0)),
    "channel_force": dict(nx=8, ny=7, nz=6, tau=0.7, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL, BC_WALL, BC_WALL),
                          force_mode=FORCE_UNIFORM, force_uniform=(1e-4, 0.0, 0.0)),
    "periodic_field": dict(nx=8, ny=8, nz=8, tau=0.55, force_mode=FORCE_FIELD),
    "mixed_lids": dict(nx=6, ny=8, nz=5, tau=0.9, bc=(BC_LID, BC_WALL, BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_LID),
                       u_lid=(0.0, 0.04, -0.01)),
}


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("name", sorted(BRUTE_CASES))
def test_oracle_equals_numpy_brute_force(q, name):
    cfg = oracle.Config(q=q, **BRUTE_CASES[name])
    F = np.zeros((3, *cfg.shape))
    if cfg.force_mode == FORCE_FIELD:
        cfg.force_field = inputs.channel_force(cfg.nx, cfg.ny, cfg.nz, seed=5, sigma=1e-4).astype(np.float64)
        F = cfg.force_field
    elif cfg.force_mode == FORCE_UNIFORM:
        F[:] = np.array(cfg.force_uniform)[:, None, None, None]
    f = noisy_equilibrium(cfg, seed=len(name) + q)
    fb = _to_brute(f, q)
    for _ in range(5):
        f = oracle.step(cfg, f)
        fb = brute.step(fb, cfg.tau, cfg.bc, cfg.u_lid, F, cfg.rho_wall)
    assert np.max(np.abs(_to_brute(f, q) - fb)) < 1e-14


@pytest.mark.parametrize("q", QS)
def test_rest_state_mass_and_momentum(q):
    cfg = oracle.Config(nx=6, ny=5, nz=4, tau=0.7, q=q)
    rho = np.full(cfg.shape, 1.03)
    u = np.zeros((3, *cfg.shape))
    u[0], u[1], u[2] = 0.04, -0.02, 0.01
    f0 = oracle.init_equilibrium(cfg, rho, u)
    assert np.max(np.abs(oracle.run(cfg, f0, 30) - f0)) < 1e-15
    cav = oracle.cavity(10, 0.6)
    cav.q = q
    g0 = oracle.init_equilibrium(cav)
    g = oracle.run(cav, g0, 60)
    assert abs(g.sum() - g0.sum()) / g0.sum() < 1e-13
    assert np.max(np.abs(oracle.moments(cav, g)[1][0])) > 1e-3
    per = oracle.Config(nx=5, ny=4, nz=3, tau=0.9, q=q, force_mode=FORCE_UNIFORM, force_uniform=(1e-4, -2e-5, 3e-5))
    r, v = inputs.random_density_velocity(per.nx, per.ny, per.nz, seed=3)
    h0 = oracle.init_equilibrium(per, r, v)
    gain = oracle.reduce(per, oracle.run(per, h0, 20))[1:4] - oracle.reduce(per, h0)[1:4]
    assert np.allclose(gain, 20 * per.n * np.array(per.force_uniform), rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("q", QS)
def test_couette_profile_exact(q):
    U, nz = 0.02, 8
    cfg = oracle.Config(nx=1, ny=1, nz=nz, tau=0.8, q=q, bc=(BC_PERIODIC,) * 4 + (BC_WALL, BC_LID),
                        u_lid=(U, 0.0, 0.0))
    f = oracle.run(cfg, oracle.init_equilibrium(cfg), 4000)
    _, u = oracle.moments(cfg, f)
    assert np.allclose(u[0, :, 0, 0], U * (np.arange(nz) + 0.5) / nz, rtol=0, atol=1e-12 * U)
    assert np.allclose(u[1:], 0.0, atol=1e-13)


def _channel(q, tau, H, F, steps):
    cfg = oracle.Config(nx=1, ny=H, nz=1, tau=tau, q=q,
                        bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL, BC_PERIODIC, BC_PERIODIC),
                        force_mode=FORCE_UNIFORM, force_uniform=(F, 0.0, 0.0))
    rho, u = oracle.moments(cfg, oracle.run(cfg, oracle.init_equilibrium(cfg), steps))
    return rho[0, :, 0], u[0, 0, :, 0]


@pytest.mark.parametrize("q", QS)
def test_poiseuille_exact_at_magic_tau(q):
    """Body-force channel between half-way walls, (tau - 1/2)^2 = 3/16: the
    walls sit exactly at y = -1/2 and H - 1/2 and the profile is the exact
    parabola u = F/(2 nu) (y + 1/2)(H - y - 1/2)."""
    tau, H, F = 0.5 + np.sqrt(3.0) / 4.0, 8, 1e-5
    rho, ux = _channel(q, tau, H, F, 3000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = F / (2.0 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.max(np.abs(ux - exact)) / np.max(exact) < 1e-10
    assert np.allclose(rho, 1.0, atol=1e-14)


@pytest.mark.parametrize("q", QS)
def test_poiseuille_curvature(q):
    """At another tau the bulk profile keeps the exact curvature -F/nu."""
    tau, H, F = 0.7, 10, 1e-5
    nu = (tau - 0.5) / 3.0
    _, ux = _channel(q, tau, H, F, int(40 * H * H / nu / 3.0) + 500)
    assert np.allclose(ux[2:] - 2.0 * ux[1:-1] + ux[:-2], -F / nu, rtol=1e-8)
    assert np.allclose(ux, ux[::-1], rtol=1e-12)


@pytest.mark.parametrize("q", QS)
def test_shear_wave_viscosity(q):
    tau = 0.8
    nu = (tau - 0.5) / 3.0

    def rate(n, steps):
        cfg = oracle.Config(nx=1, ny=n, nz=1, tau=tau, q=q)
        f = oracle.init_equilibrium(cfg, None, inputs.shear_wave_velocity(1, n, 1, 1e-4, axis_u=0, axis_k=1))
        f = oracle.run(cfg, f, steps[0])
        a0 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
        f = oracle.run(cfg, f, steps[1] - steps[0])
        a1 = np.max(np.abs(oracle.moments(cfg, f)[1][0]))
        return -np.log(a1 / a0) / ((2.0 * np.pi / n) ** 2 * (steps[1] - steps[0]))

    e32 = abs(rate(32, (60, 260)) / nu - 1.0)
    e64 = abs(rate(64, (240, 1040)) / nu - 1.0)
    assert e32 < 1e-2
    assert e64 < 0.35 * e32 + 1e-6


def test_mrt_is_d3q19_only():
    with pytest.raises(ValueError):
        oracle.Config(nx=4, ny=4, nz=4, tau=0.7, q=27, collision=oracle.COLL_MRT)
    with pytest.raises(ValueError):
        oracle.Config(nx=4, ny=4, nz=4, tau=0.7, q=21)
