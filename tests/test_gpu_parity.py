"""GPU path against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative max-norm, max|a - b| / max|b|):
  FP64 storage: 1e-12 on populations and velocities (the kernels evaluate
                the same formulas in the shifted form f - w, a different
                rounding order from the oracle's).
  FP32 storage: 1e-5 on velocities after 100 steps of the 32^3 cavity.
"""
import numpy as np
import pytest

import oracle
from gpu_cases import (cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32,
                       start_state)
from helpers import relmax

pytestmark = pytest.mark.gpu

CASES = cases()
VARIANTS = ["two_lattice", "aa", "merged", "merged_snapshot", "wavefront"]


def _variant(v):
    """(variant, tile): "merged" takes the automatic tiles (the shadow-shell
    sweep where z is not periodic), "merged_snapshot" an explicit 32 x 4 tile
    (the snapshot sweep)."""
    return ("merged", (32, 4)) if v == "merged_snapshot" else (v, (0, 0))


@pytest.mark.parametrize("variant", VARIANTS)
def test_cavity_32_fp64_100_steps(gpu, variant):
    """32^3 lid-driven cavity, FP64, tau = 0.6, lid 0.05 on z+, at rest, 100 steps."""
    cfg = oracle.cavity(32, 0.6)
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    rho_r, u_r = oracle.moments(cfg, ref)
    v, tile = _variant(variant)
    lat = make_gpu(cfg, "f64", v, tile=tile)
    lat.init_equilibrium()
    lat.step(100)
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12
    assert relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("storage", ["f32", "f32s"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_cavity_32_fp32_100_steps(gpu, storage, variant):
    cfg = oracle.cavity(32, 0.6)
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    _, u_r = oracle.moments(cfg, ref)
    v, tile = _variant(variant)
    if storage != "f64" and v == "merged" and tile != (0, 0):
        tile = (32, 16)
    lat = make_gpu(cfg, storage, v, tile=tile)
    lat.init_equilibrium()
    lat.step(100)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nsteps", [1, 4, 7])
def test_fp64_cases(gpu, name, variant, nsteps):
    cfg = oracle_force_as_f32(CASES[name])
    f0 = start_state(cfg, seed=nsteps)
    ref = oracle.run(cfg, f0, nsteps)
    v, tile = _variant(variant)
    lat = make_gpu(cfg, "f64", v, tile=tile)
    load_state(lat, f0)
    lat.step(nsteps)
    assert lat.time == nsteps
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho_r, u_r = oracle.moments(cfg, ref)
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12
    assert relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nsteps", [2, 3])
def test_reduce_fp64(gpu, name, nsteps):
    cfg = oracle_force_as_f32(CASES[name])
    f0 = start_state(cfg, seed=5)
    ref = oracle.run(cfg, f0, nsteps)
    lat = make_gpu(cfg, "f64", "aa")
    load_state(lat, f0)
    lat.step(nsteps)          # odd nsteps leaves the AA state at the other parity
    got = lat.reduce()
    exp = oracle.reduce(cfg, ref)
    assert abs(got[0] - exp[0]) <= 1e-13 * abs(exp[0])
    scale = max(np.max(np.abs(exp[1:4])), 1e-300)
    assert np.max(np.abs(got[1:4] - exp[1:4])) <= 1e-11 * scale + 1e-15
    assert abs(got[4] - exp[4]) <= 1e-11 * abs(exp[4]) + 1e-18


def test_reduce_flags_nonfinite(gpu):
    import torch
    from paper_2208_05429_gb300.lbm import LBM_ENONFINITE, LbmError
    cfg = oracle.cavity(12, 0.6)
    f0 = start_state(cfg)
    f0[3, 4, 5, 6] = np.nan
    lat = make_gpu(cfg, "f32", "aa")
    load_state(lat, f0)
    with pytest.raises(LbmError) as ei:
        lat.reduce()
    assert ei.value.status == LBM_ENONFINITE
    lat2 = make_gpu(cfg, "f32", "aa")
    load_state(lat2, start_state(cfg))
    assert np.all(np.isfinite(lat2.reduce()))


@pytest.mark.parametrize("variant", ["merged", "wavefront"])
def test_sampled_step_at_bench_size(gpu, variant):
    """256^3 cavity (the benchmark workload, FP32, default launch shapes):
    after 20 steps, one more GPU step is checked on 400 sampled cells against
    the oracle stepping those cells alone from the GPU's own state."""
    import torch
    from paper_2208_05429_gb300 import inputs
    n = 256
    cfg = oracle.cavity(n, 0.55)
    lat = make_gpu(cfg, "f32", variant)
    lat.init_equilibrium()
    lat.step(20)
    f20 = gpu_state(lat)                       # oracle order, float64
    lat.step(1)
    f21 = lat.populations(torch.float32)
    cells = inputs.sample_cells(n, n, n, 400, seed=11)
    # force edge and corner cells into the sample
    cells[:8] = [[0, 0, 0], [n - 1, n - 1, n - 1], [0, n - 1, n - 1], [n - 1, 0, n - 1],
                 [5, 0, n - 1], [n - 1, 7, 0], [0, 9, 3], [17, n - 1, n - 2]]
    exp = oracle.step_cells(cfg, f20, cells)
    from gpu_cases import to_oracle_order
    got = np.stack([to_oracle_order(f21[:, z, y, x].cpu().numpy().astype(np.float64)) for x, y, z in cells])
    assert relmax(got, exp) <= 2e-7
    del f20


@pytest.mark.parametrize("variant", ["merged", "wavefront"])
def test_mass_conservation_bench_size(gpu, variant):
    """Exact mass conservation of the cavity holds at 256^3 (FP64 sums of an
    FP32 lattice: drift only from storage rounding)."""
    cfg = oracle.cavity(256, 0.55)
    lat = make_gpu(cfg, "f32s", variant)
    lat.init_equilibrium()
    m0 = lat.reduce()[0]
    lat.step(100)
    m1 = lat.reduce()[0]
    assert abs(m1 - m0) / m0 <= 1e-7
