"""The TRT collision on the GPU (AA and TWO_LATTICE schedules) against the
FP64 oracle's TRT, through the C ABI.

Tolerances as for BGK (relative max-norm): FP64 1e-12 on populations and
velocities; FP32 1e-5 on velocities after 100 steps of the 32^3 cavity."""
import numpy as np
import pytest

import oracle
from gpu_cases import cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state
from helpers import relmax

pytestmark = pytest.mark.gpu

TRT_CASES = ["channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "narrow_2x21x5", "flat_40x35x1"]


def _trt(cfg, lam):
    cfg.collision = oracle.COLL_TRT
    cfg.trt_lambda = lam
    return cfg


@pytest.mark.parametrize("name", TRT_CASES)
@pytest.mark.parametrize("variant", ["aa", "two_lattice"])
@pytest.mark.parametrize("lam", [3.0 / 16.0, 0.05])
@pytest.mark.parametrize("nsteps", [1, 4, 7])
def test_trt_fp64_cases(gpu, name, variant, lam, nsteps):
    cfg = _trt(oracle_force_as_f32(cases()[name]), lam)
    f0 = start_state(cfg, seed=nsteps + 30)
    ref = oracle.run(cfg, f0, nsteps)
    lat = make_gpu(cfg, "f64", variant)
    load_state(lat, f0)
    lat.step(nsteps)
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho_r, u_r = oracle.moments(cfg, ref)
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12 and relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("storage", ["f32", "f32s"])
def test_trt_cavity_32_fp32_100_steps(gpu, storage):
    cfg = _trt(oracle.cavity(32, 0.6), 3.0 / 16.0)
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    _, u_r = oracle.moments(cfg, ref)
    lat = make_gpu(cfg, storage, "aa")
    lat.init_equilibrium()
    lat.step(100)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_trt_aa_equals_two_lattice(gpu, storage):
    import torch
    cfg = _trt(oracle_force_as_f32(cases()["channel_37x19x23"]), 0.1)
    f0 = start_state(cfg, seed=5)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f0)
    a.step(9)
    t = make_gpu(cfg, storage, "two_lattice")
    load_state(t, f0)
    t.step(9)
    assert torch.equal(a.populations(torch.float64), t.populations(torch.float64))


def test_trt_poiseuille_exact_on_gpu(gpu):
    """Body-force channel, walls in y, tau = 1.2, Lambda = 3/16, FP64 on the
    GPU: the steady profile is the exact parabola (the oracle's pin, run by
    the CUDA kernels)."""
    from oracle import BC_PERIODIC, BC_WALL, FORCE_UNIFORM
    tau, H, F = 1.2, 8, 1e-5
    cfg = oracle.Config(nx=3, ny=H, nz=2, tau=tau, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL,
                                                       BC_PERIODIC, BC_PERIODIC),
                        force_mode=FORCE_UNIFORM, force_uniform=(F, 0.0, 0.0))
    cfg = _trt(cfg, 3.0 / 16.0)
    lat = make_gpu(cfg, "f64", "aa")
    lat.init_equilibrium()
    nu = (tau - 0.5) / 3.0
    lat.step(int(60 * H * H / nu / 3.0) + 1000)
    _, u = gpu_moments(lat)
    y = np.arange(H)
    exact = F / (2.0 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.max(np.abs(u[0, 0, :, 1] - exact)) / np.max(exact) < 1e-9


@pytest.mark.parametrize("storage", ["f32", "f16s"])
@pytest.mark.parametrize("name", ["cavity16", "mixed_33x40x9", "channel_37x19x23"])
def test_trt_merged_equals_aa(gpu, monkeypatch, storage, name):
    """MERGED with TRT: the neighbour-synchronised sweep where it runs (the
    walled cavity), else the AA pair (the shadow-shell sweep is BGK only);
    bit-identical to AA either way, including an odd step count."""
    import torch
    cfg = _trt(oracle_force_as_f32(cases()[name]), 0.1)
    f0 = start_state(cfg, seed=7)
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
