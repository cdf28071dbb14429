"""Pins of the oracle's lattice table, equilibrium and collision against the
closed-form identities of the D3Q19 lattice and of the BGK + Guo operator."""
import itertools

import numpy as np
import pytest

import oracle


def test_velocity_set_is_d3q19():
    c, w, opp = oracle.lattice()
    vecs = {tuple(v) for v in c}
    expected = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2}
    assert vecs == expected and len(c) == 19
    for i in range(19):
        n2 = int((c[i] ** 2).sum())
        assert w[i] == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[n2]


def test_swap_ordering_and_opposites():
    """Directions 1..9: first non-zero component -1 (the swap half, Sec. 3);
    i+9 opposite of i."""
    c, _, opp = oracle.lattice()
    assert tuple(c[0]) == (0, 0, 0)
    for i in range(1, 10):
        first = next(v for v in c[i] if v != 0)
        assert first == -1
        assert np.array_equal(c[i + 9], -c[i])
        assert opp[i] == i + 9 and opp[i + 9] == i
    assert opp[0] == 0


def test_lattice_moment_isotropy():
    c, w, _ = oracle.lattice()
    cf = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("q,qa->a", w, cf), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, cf, cf), np.eye(3) / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, cf, cf, cf), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("q,qa,qb,qc,qd->abcd", w, cf, cf, cf, cf), iso4, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """feq reproduces rho, rho u and rho u u + rho/3 I exactly (to rounding)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rng.uniform(-0.2, 0.2)
    u = rng.uniform(-0.1, 0.1, size=3)
    feq = oracle.equilibrium(rho, u)
    c, _, _ = oracle.lattice()
    cf = c.astype(np.float64)
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(cf.T @ feq, rho * u, atol=1e-15)
    P = np.einsum("q,qa,qb->ab", feq, cf, cf)
    assert np.allclose(P, rho * np.outer(u, u) + rho / 3.0 * np.eye(3), atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_collision_invariants(seed):
    """BGK + Guo: mass kept; momentum gains exactly F; the non-equilibrium
    part relaxes by (1 - omega) when F = 0; feq is a fixed point."""
    rng = np.random.default_rng(100 + seed)
    c, w, _ = oracle.lattice()
    cf = c.astype(np.float64)
    tau = rng.uniform(0.51, 2.0)
    f = w * (1.0 + rng.uniform(-0.3, 0.3, size=19))
    F = rng.uniform(-1e-3, 1e-3, size=3)
    fs = oracle.collide_cell(tau, f, F)
    assert abs(fs.sum() - f.sum()) < 1e-15
    assert np.allclose(cf.T @ fs, cf.T @ f + F, atol=1e-16)
    # F = 0: f* - feq = (1 - omega)(f - feq) with feq of the pre-collision moments
    fs0 = oracle.collide_cell(tau, f)
    rho = f.sum()
    u = (cf.T @ f) / rho
    feq = oracle.equilibrium(rho, u)
    assert np.allclose(fs0 - feq, (1.0 - 1.0 / tau) * (f - feq), atol=1e-16)
    assert np.allclose(oracle.collide_cell(tau, feq), feq, atol=1e-16)


def test_guo_force_second_moment():
    """The Guo source adds (1 - omega/2)(u F + F u) to the momentum flux,
    the term that makes the scheme second-order with a body force."""
    rng = np.random.default_rng(7)
    c, w, _ = oracle.lattice()
    cf = c.astype(np.float64)
    tau = 0.8
    om = 1.0 / tau
    u0 = rng.uniform(-0.05, 0.05, size=3)
    F = rng.uniform(-1e-3, 1e-3, size=3)
    # choose f = feq(rho, u) with u the force-corrected velocity of f itself:
    # sum f c = rho u - F/2 so that (sum f c + F/2)/rho = u
    feq = oracle.equilibrium(1.0, u0)
    # shift the momentum by -F/2 with a perturbation of zero mass and zero stress
    f = feq - 1.5 * w * (cf @ F)
    fs = oracle.collide_cell(tau, f, F)
    # the equilibrium part of the update is exact here; the flux change is
    # -omega (P(f) - P(feq)) + (1 - omega/2) (u F + F u)
    P = lambda g: np.einsum("q,qa,qb->ab", g, cf, cf)  # noqa: E731
    expected = P(f) - om * (P(f) - P(feq)) + (1.0 - 0.5 * om) * (np.outer(u0, F) + np.outer(F, u0))
    assert np.allclose(P(fs), expected, atol=1e-15)


def test_oracle_result_independent_of_threads():
    """The host timing runs the oracle on one thread and on all of them; every
    cell is computed the same way, so the states are bitwise equal."""
    cfg = oracle.cavity(12, 0.6)
    f0 = oracle.init_equilibrium(cfg)
    before = oracle.threads()
    try:
        oracle.threads(1)
        one = oracle.run(cfg, f0.copy(), 5)
        oracle.threads(max(2, before))
        many = oracle.run(cfg, f0.copy(), 5)
    finally:
        oracle.threads(before)
    assert np.array_equal(one, many)
