"""The multiple-relaxation-time collision (Hermite moments; orders up to
two at 1/tau, order three at s3, order four at s4) on the GPU against the
FP64 oracle's, through the C ABI, on every schedule.

Tolerances as for BGK (relative max-norm): FP64 1e-12 on populations and
velocities; FP32 1e-5 on velocities after 100 steps of the 32^3 cavity."""
import pytest

import oracle
from gpu_cases import cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state
from helpers import relmax

pytestmark = pytest.mark.gpu

MRT_CASES = ["channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "narrow_2x21x5", "flat_40x35x1"]


def _mrt(cfg, s3=1.3, s4=1.7):
    cfg.collision = oracle.COLL_MRT
    cfg.mrt_s3, cfg.mrt_s4 = s3, s4
    return cfg


@pytest.mark.parametrize("name", MRT_CASES)
@pytest.mark.parametrize("variant", ["aa", "two_lattice", "merged"])
@pytest.mark.parametrize("rates", [(1.3, 1.7), (0.8, 1.95)])
def test_mrt_fp64_cases(gpu, name, variant, rates):
    cfg = _mrt(oracle_force_as_f32(cases()[name]), *rates)
    f0 = start_state(cfg, seed=50)
    ref = oracle.run(cfg, f0, 5)
    lat = make_gpu(cfg, "f64", variant)
    load_state(lat, f0)
    lat.step(5)
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho_r, u_r = oracle.moments(cfg, ref)
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12 and relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("storage", ["f32", "f32s"])
def test_mrt_cavity_32_fp32_100_steps(gpu, storage):
    cfg = _mrt(oracle.cavity(32, 0.6))
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    _, u_r = oracle.moments(cfg, ref)
    lat = make_gpu(cfg, storage, "aa")
    lat.init_equilibrium()
    lat.step(100)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("name", ["cavity16", "channel_37x19x23"])
def test_mrt_schedules_bitwise_equal(gpu, monkeypatch, storage, name):
    """AA, TWO_LATTICE and MERGED (the neighbour-synchronised sweep on the
    walled cavity, the AA pair elsewhere) agree bit for bit."""
    import torch
    cfg = _mrt(oracle_force_as_f32(cases()[name]))
    f0 = start_state(cfg, seed=12)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f0)
    a.step(7)
    want = a.populations(torch.float64)
    t = make_gpu(cfg, storage, "two_lattice")
    load_state(t, f0)
    t.step(7)
    assert torch.equal(t.populations(torch.float64), want)
    monkeypatch.setenv("LBM_MERGED_SWEEP", "neighbour")
    m = make_gpu(cfg, storage, "merged")
    monkeypatch.delenv("LBM_MERGED_SWEEP")
    load_state(m, f0)
    m.profile(True)
    m.step(7)
    ran = m.profile_read()
    m.profile(False)
    if name == "cavity16":
        assert "merged" in ran, ran
    assert torch.equal(m.populations(torch.float64), want)
