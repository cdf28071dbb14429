"""The paper's own CPU algorithms (cpu_memaware: Alg. 1 fused swap, Alg. 2
sequential two-step prism, Alg. 3 OpenMP two-step prism) against the oracle
and against each other.

The paper verifies that its two-step solvers reproduce the single-step one
(Sec. 5.1).  Here:
  * Alg. 1 equals the FP64 oracle to 1e-14 relative max-norm (same formulas,
    a different direction order in the sums: last-bit differences only);
  * Alg. 2 (every prism stride, with and without prisms) and Alg. 3 (1 to 4
    threads, several strides) equal Alg. 1 bit for bit;
  * every traversal runs through the dependency checker, which counts each
    collision made before all its inputs were streamed and each link
    exchanged before both its cells collided, or twice: zero violations;
  * the checker itself catches a planted ordering mistake.
"""
import numpy as np
import pytest

import cpu_memaware as cm
import oracle
from helpers import relmax

WALL, LID = oracle.BC_WALL, oracle.BC_LID


def _perm():
    """k-th direction of cpu_memaware = direction perm[k] of the oracle."""
    c_m, _ = cm.lattice()
    c_o, _, _ = oracle.lattice()
    idx = {tuple(int(a) for a in v): k for k, v in enumerate(c_o)}
    return [idx[tuple(int(a) for a in v)] for v in c_m]


def _pair(nx, ny, nz, tau=0.6, bc=(WALL, WALL, WALL, WALL, WALL, LID), u_lid=(0.05, 0.0, 0.0), force=None):
    kw = {}
    if force is not None:
        kw = dict(force_mode=oracle.FORCE_UNIFORM, force_uniform=tuple(force))
    ocfg = oracle.Config(nx=nx, ny=ny, nz=nz, tau=tau, bc=tuple(bc), u_lid=tuple(u_lid), **kw)
    mcfg = cm.Config(nx, ny, nz, tau, bc=tuple(bc), u_lid=tuple(u_lid), force_uniform=force)
    return ocfg, mcfg


def _start(ocfg, seed):
    rng = np.random.default_rng(seed)
    f = oracle.init_equilibrium(ocfg)
    return f * (1.0 + 0.02 * rng.standard_normal(f.shape))


SHAPES = [
    dict(nx=8, ny=8, nz=8),
    dict(nx=13, ny=9, nz=11, bc=(LID, WALL, WALL, WALL, WALL, LID), u_lid=(0.0, 0.03, 0.02),
         force=(1e-5, -2e-5, 3e-6)),
    dict(nx=5, ny=7, nz=12, bc=(WALL, WALL, LID, WALL, WALL, WALL), u_lid=(0.04, 0.0, -0.01)),
    dict(nx=17, ny=4, nz=16),
    dict(nx=3, ny=3, nz=3),
]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_fuse_matches_oracle(shape, nsteps):
    ocfg, mcfg = _pair(**SHAPES[shape])
    f0 = _start(ocfg, seed=shape)
    perm = _perm()
    ref = oracle.run(ocfg, f0, nsteps)
    cm.reset_violations()
    got = cm.run("fuse", mcfg, f0[perm], nsteps, checked=True)
    assert cm.violations() == 0
    assert relmax(got, ref[perm]) <= 1e-14


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("tile", [1, 2, 3, 5, 8, 0])
def test_two_step_prism_equals_fuse(shape, tile):
    """Alg. 2: two sweeps (four steps) and an odd count (a last Alg. 1 step)."""
    ocfg, mcfg = _pair(**SHAPES[shape])
    f0 = _start(ocfg, seed=10 + shape)[_perm()]
    for nsteps in (4, 3):
        want = cm.run("fuse", mcfg, f0, nsteps)
        cm.reset_violations()
        got = cm.run("two_step", mcfg, f0, nsteps, tile=tile, checked=True)
        assert cm.violations() == 0, (tile, nsteps)
        assert np.array_equal(got, want), (tile, nsteps)
        assert np.array_equal(cm.run("two_step", mcfg, f0, nsteps, tile=tile), want)


@pytest.mark.parametrize("nx,ny,nz", [(1, 6, 9), (6, 1, 9), (7, 5, 1), (2, 2, 2), (1, 1, 4)])
def test_two_step_prism_degenerate_shapes(nx, ny, nz):
    ocfg, mcfg = _pair(nx, ny, nz)
    f0 = _start(ocfg, seed=3)[_perm()]
    want = cm.run("fuse", mcfg, f0, 2)
    for tile in (1, 2, 0):
        cm.reset_violations()
        assert np.array_equal(cm.run("two_step", mcfg, f0, 2, tile=tile, checked=True), want)
        assert cm.violations() == 0


@pytest.mark.parametrize("shape", [0, 1, 3])
@pytest.mark.parametrize("nthreads", [1, 2, 3, 4])
@pytest.mark.parametrize("tile", [2, 4, 0])
def test_two_step_prism_omp_equals_fuse(shape, nthreads, tile):
    """Alg. 3 with X-slabs of at least three layers (16 layers: up to 4
    threads, uneven slabs included)."""
    ocfg, mcfg = _pair(**SHAPES[shape])
    f0 = _start(ocfg, seed=20 + shape)[_perm()]
    want = cm.run("fuse", mcfg, f0, 4)
    cm.reset_violations()
    got = cm.run("omp", mcfg, f0, 4, tile=tile, nthreads=nthreads, checked=True)
    assert cm.violations() == 0
    assert np.array_equal(got, want)
    assert np.array_equal(cm.run("omp", mcfg, f0, 4, tile=tile, nthreads=nthreads), want)


def test_cavity_32_all_algorithms():
    """The paper's verification case in small: a 32^3 lid-driven cavity from
    rest, 6 steps, every algorithm equal to Alg. 1, Alg. 1 equal to the
    oracle."""
    ocfg, mcfg = _pair(32, 32, 32, tau=0.55)
    perm = _perm()
    f0 = oracle.init_equilibrium(ocfg)
    ref = oracle.run(ocfg, f0, 6)[perm]
    want = cm.run("fuse", mcfg, f0[perm], 6)
    assert relmax(want, ref) <= 1e-14
    for tile in (8, 16, 0):
        assert np.array_equal(cm.run("two_step", mcfg, f0[perm], 6, tile=tile), want)
        cm.reset_violations()
        assert np.array_equal(cm.run("omp", mcfg, f0[perm], 6, tile=tile, nthreads=4, checked=True), want)
        assert cm.violations() == 0


def test_checker_catches_planted_misorder():
    """One step of Alg. 1 with its inner-cell stage run before the box cells
    have collided: the checker must count violations (else a zero count above
    would mean nothing)."""
    ocfg, mcfg = _pair(8, 7, 6)
    assert cm.planted_misorder(mcfg, _start(ocfg, seed=1)[_perm()]) > 0


def test_invalid_configurations_rejected():
    ocfg, mcfg = _pair(8, 8, 8)
    f0 = _start(ocfg, seed=2)[_perm()]
    per = cm.Config(8, 8, 8, 0.6, bc=(0, 0, WALL, WALL, WALL, LID))
    with pytest.raises(ValueError):
        cm.run("fuse", per, f0, 1)
    with pytest.raises(ValueError):
        cm.run("fuse", cm.Config(8, 8, 8, 0.5), f0, 1)
    ocfg2, mcfg2 = _pair(8, 8, 2)
    with pytest.raises(ValueError):   # Alg. 3 needs three layers per slab
        cm.run("omp", mcfg2, _start(ocfg2, seed=2)[_perm()], 2)
    ocfg3, mcfg3 = _pair(1, 8, 8)
    with pytest.raises(ValueError):   # and two rows and columns per layer
        cm.run("omp", mcfg3, _start(ocfg3, seed=2)[_perm()], 2)
