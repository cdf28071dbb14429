"""The regularised BGK collision on the GPU (AA and TWO_LATTICE schedules)
against the FP64 oracle's regularised collision, through the C ABI.

Tolerances as for BGK (relative max-norm): FP64 1e-12 on populations and
velocities; FP32 1e-5 on velocities after 100 steps of the 32^3 cavity."""
import pytest

import oracle
from gpu_cases import cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state
from helpers import relmax

pytestmark = pytest.mark.gpu

REG_CASES = ["channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "narrow_2x21x5", "flat_40x35x1"]


def _reg(cfg):
    cfg.collision = oracle.COLL_REG
    return cfg


@pytest.mark.parametrize("name", REG_CASES)
@pytest.mark.parametrize("variant", ["aa", "two_lattice"])
@pytest.mark.parametrize("nsteps", [1, 4, 7])
def test_reg_fp64_cases(gpu, name, variant, nsteps):
    cfg = _reg(oracle_force_as_f32(cases()[name]))
    f0 = start_state(cfg, seed=nsteps + 40)
    ref = oracle.run(cfg, f0, nsteps)
    lat = make_gpu(cfg, "f64", variant)
    load_state(lat, f0)
    lat.step(nsteps)
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho_r, u_r = oracle.moments(cfg, ref)
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12 and relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("storage", ["f32", "f32s"])
def test_reg_cavity_32_fp32_100_steps(gpu, storage):
    cfg = _reg(oracle.cavity(32, 0.6))
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    _, u_r = oracle.moments(cfg, ref)
    lat = make_gpu(cfg, storage, "aa")
    lat.init_equilibrium()
    lat.step(100)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_reg_aa_equals_two_lattice(gpu, storage):
    import torch
    cfg = _reg(oracle_force_as_f32(cases()["channel_37x19x23"]))
    f0 = start_state(cfg, seed=6)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f0)
    a.step(9)
    t = make_gpu(cfg, storage, "two_lattice")
    load_state(t, f0)
    t.step(9)
    assert torch.equal(a.populations(torch.float64), t.populations(torch.float64))


def test_reg_differs_from_bgk_on_gpu(gpu):
    """The GPU runs the regularised operator, not BGK: from a noisy start the
    two states differ by far more than rounding after a few steps."""
    cfg = oracle_force_as_f32(cases()["channel_37x19x23"])
    f0 = start_state(cfg, seed=8)
    lat_b = make_gpu(cfg, "f64", "aa")
    load_state(lat_b, f0)
    lat_b.step(3)
    lat_r = make_gpu(_reg(oracle_force_as_f32(cases()["channel_37x19x23"])), "f64", "aa")
    load_state(lat_r, f0)
    lat_r.step(3)
    assert relmax(gpu_state(lat_r), gpu_state(lat_b)) > 1e-6


@pytest.mark.parametrize("storage", ["f32", "f16s"])
@pytest.mark.parametrize("name", ["cavity16", "mixed_33x40x9", "channel_37x19x23"])
def test_reg_merged_equals_aa(gpu, monkeypatch, storage, name):
    """MERGED with the regularised collision: the neighbour-synchronised
    sweep where it runs (the walled cavity), else the AA pair; bit-identical
    to AA either way, including an odd step count."""
    import torch
    cfg = _reg(oracle_force_as_f32(cases()[name]))
    f0 = start_state(cfg, seed=9)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f0)
    a.step(7)
    for sweep in ("neighbour", "shadow"):
        monkeypatch.setenv("LBM_MERGED_SWEEP", sweep)
        m = make_gpu(cfg, storage, "merged")
        monkeypatch.delenv("LBM_MERGED_SWEEP")
        load_state(m, f0)
        m.profile(True)
        m.step(7)
        ran = m.profile_read()
        m.profile(False)
        if name == "cavity16" and sweep == "neighbour":
            assert "merged" in ran, ran
        assert torch.equal(m.populations(torch.float64), a.populations(torch.float64)), (sweep, ran)


def test_reg_merged_fp64_against_oracle(gpu):
    """FP64 MERGED with the regularised collision (the AA pair: FP64 has no
    neighbour-synchronised sweep) against the oracle, 1e-12."""
    cfg = _reg(oracle_force_as_f32(cases()["mixed_33x40x9"]))
    f0 = start_state(cfg, seed=11)
    ref = oracle.run(cfg, f0, 6)
    lat = make_gpu(cfg, "f64", "merged")
    load_state(lat, f0)
    lat.step(6)
    assert relmax(gpu_state(lat), ref) <= 1e-12
