"""The D3Q15 and D3Q27 kernels on the GPU (TWO_LATTICE, AA, and MERGED,
which runs the AA pair on these lattices) against the FP64 oracle's D3Q15 /
D3Q27 update, through the C ABI.

Tolerances as for D3Q19: FP64 storage 1e-12 relative max-norm on
populations and moments; FP32 storage 1e-5 on velocities after 100 steps of
the 32^3 cavity; 16-bit storage within one storage ulp (+4e-8) per step of
the oracle's step followed by the storage rounding; the full 256^3 lattice
in FP32 within the 1.5e-7 of the D3Q19 check after one even and one odd
step.  The schedules agree bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import BC_PERIODIC, BC_WALL, FORCE_UNIFORM
from gpu_cases import cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state
from helpers import relmax

pytestmark = pytest.mark.gpu

QS = [15, 27]
NAMES = ["cavity16", "channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "flat_40x35x1",
         "narrow_2x21x5", "pencil_1x19x4", "periodic_33x15x2"]


def _case(name, q, collision=oracle.COLL_BGK, lam=3.0 / 16.0):
    cfg = oracle_force_as_f32(cases()[name])
    cfg.q = q
    cfg.collision = collision
    cfg.trt_lambda = lam
    return cfg


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("variant", ["two_lattice", "aa", "merged"])
@pytest.mark.parametrize("nsteps", [1, 4, 7])
def test_fp64_cases(gpu, q, name, variant, nsteps):
    cfg = _case(name, q)
    f0 = start_state(cfg, seed=nsteps + q)
    ref = oracle.run(cfg, f0, nsteps)
    lat = make_gpu(cfg, "f64", variant)
    load_state(lat, f0)
    lat.step(nsteps)
    assert lat.time == nsteps
    assert relmax(gpu_state(lat), ref) <= 1e-12
    rho_r, u_r = oracle.moments(cfg, ref)
    rho, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-12 and relmax(rho, rho_r) <= 1e-12


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("collision", [oracle.COLL_TRT, oracle.COLL_REG])
@pytest.mark.parametrize("name", ["channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9"])
@pytest.mark.parametrize("variant", ["two_lattice", "aa"])
def test_other_collisions_fp64(gpu, q, collision, name, variant):
    cfg = _case(name, q, collision, lam=0.1)
    f0 = start_state(cfg, seed=40 + q)
    ref = oracle.run(cfg, f0, 5)
    lat = make_gpu(cfg, "f64", variant)
    load_state(lat, f0)
    lat.step(5)
    assert relmax(gpu_state(lat), ref) <= 1e-12


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("storage", ["f32", "f32s"])
@pytest.mark.parametrize("variant", ["two_lattice", "aa"])
def test_cavity_32_fp32_100_steps(gpu, q, storage, variant):
    cfg = oracle.cavity(32, 0.6)
    cfg.q = q
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 100)
    _, u_r = oracle.moments(cfg, ref)
    lat = make_gpu(cfg, storage, variant)
    lat.init_equilibrium()
    lat.step(100)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("storage", ["f32", "f32s", "f16s", "bf16s"])
@pytest.mark.parametrize("name", ["cavity16", "channel_37x19x23", "mixed_33x40x9"])
def test_schedules_bitwise_equal(gpu, q, storage, name):
    import torch
    cfg = _case(name, q)
    f0 = start_state(cfg, seed=7)
    out = {}
    for variant in ("two_lattice", "aa", "merged"):
        lat = make_gpu(cfg, storage, variant)
        load_state(lat, f0)
        lat.step(9)
        out[variant] = lat.populations(torch.float64)
    assert torch.equal(out["aa"], out["two_lattice"]) and torch.equal(out["merged"], out["aa"])


def _ulp(s, storage):
    a = np.abs(s)
    if storage == "f16s":
        u = np.spacing(a.astype(np.float16)).astype(np.float64)
    else:
        _, e = np.frexp(a)
        u = np.ldexp(1.0, e - 8)
    return np.maximum(u, 2.0 ** -133)


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("name", ["channel_37x19x23", "mixed_33x40x9"])
def test_16bit_steps_within_one_storage_ulp(gpu, q, storage, name):
    """One AA even and one odd step, each against the oracle stepping the
    GPU's own state once and rounding to the storage format."""
    _, w, _ = oracle.lattice(q)
    w32 = w.astype(np.float32)[:, None, None, None]
    cfg = _case(name, q)
    f0, _ = oracle.store_round(start_state(cfg, seed=21), storage)
    lat = make_gpu(cfg, storage, "aa")
    load_state(lat, f0)
    prev = f0
    for _ in (1, 2):
        lat.step(1)
        _, s_exp = oracle.store_round(oracle.run(cfg, prev, 1), storage)
        got = gpu_state(lat)
        diff = np.abs(got - (s_exp.astype(np.float32) + w32).astype(np.float64))
        assert np.all(diff <= _ulp(s_exp, storage) + 4e-8)
        assert np.mean(diff == 0.0) >= 0.99
        prev = got


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("nsteps", [2, 3])
def test_reduce_fp64(gpu, q, nsteps):
    cfg = _case("channel_37x19x23", q)
    f0 = start_state(cfg, seed=5)
    ref = oracle.run(cfg, f0, nsteps)
    lat = make_gpu(cfg, "f64", "aa")
    load_state(lat, f0)
    lat.step(nsteps)       # odd nsteps leaves the AA state at the other parity
    got, exp = lat.reduce(), oracle.reduce(cfg, ref)
    assert abs(got[0] - exp[0]) <= 1e-13 * abs(exp[0])
    assert np.max(np.abs(got[1:4] - exp[1:4])) <= 1e-11 * np.max(np.abs(exp[1:4])) + 1e-15
    assert abs(got[4] - exp[4]) <= 1e-11 * abs(exp[4]) + 1e-18


@pytest.mark.parametrize("q", QS)
def test_equilibrium_init_matches_oracle(gpu, q):
    import torch
    from paper_2208_05429_gb300 import inputs
    cfg = oracle.Config(nx=20, ny=12, nz=9, tau=0.7, q=q)
    rho, u = inputs.random_density_velocity(cfg.nx, cfg.ny, cfg.nz, seed=9)
    ref = oracle.init_equilibrium(cfg, rho, u)
    lat = make_gpu(cfg, "f64", "aa")
    lat.init_equilibrium(torch.tensor(rho, device=lat.device), torch.tensor(u, device=lat.device))
    assert relmax(gpu_state(lat), ref) <= 1e-15


@pytest.mark.parametrize("q", QS)
def test_poiseuille_exact_on_gpu(gpu, q):
    """Body-force channel between half-way walls at (tau - 1/2)^2 = 3/16, FP64:
    the GPU reaches the exact parabola (the oracle's pin, run by the kernels)."""
    tau, H, F = 0.5 + np.sqrt(3.0) / 4.0, 8, 1e-5
    cfg = oracle.Config(nx=3, ny=H, nz=2, tau=tau, q=q, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL,
                                                              BC_PERIODIC, BC_PERIODIC),
                        force_mode=FORCE_UNIFORM, force_uniform=(F, 0.0, 0.0))
    lat = make_gpu(cfg, "f64", "aa")
    lat.init_equilibrium()
    lat.step(3000)
    _, u = gpu_moments(lat)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = F / (2.0 * nu) * (y + 0.5) * (H - y - 0.5)
    assert np.max(np.abs(u[0, 0, :, 1] - exact)) / np.max(exact) < 1e-10


def test_unsupported_combinations(gpu):
    import torch
    from paper_2208_05429_gb300.lbm import LBM_EUNSUPPORTED, Lattice, LbmError
    with pytest.raises(LbmError) as ei:
        Lattice((8, 8, 8), 0.7, collision="mrt", lattice=27)
    assert ei.value.status == LBM_EUNSUPPORTED
    lat = Lattice((8, 8, 8), 0.7, lattice=15, storage="f64")
    lat.init_equilibrium()
    with pytest.raises(LbmError) as ei:
        lat.adjoint_forward(4, 2)
    assert ei.value.status == LBM_EUNSUPPORTED
    assert lat.populations(torch.float64).shape == (15, 8, 8, 8)


@pytest.mark.parametrize("q", QS)
def test_full_lattice_aa_steps_at_bench_size(gpu, q):
    """The 256^3 cavity (tau = 0.55, FP32): after 20 steps, one AA even and
    one odd step over the whole lattice, each against one FP64 oracle step
    from the GPU's own state."""
    from paper_2208_05429_gb300.lbm import CAVITY_BC, Lattice
    cfg = oracle.cavity(256, 0.55)
    cfg.q = q
    lat = Lattice((256, 256, 256), 0.55, bc=CAVITY_BC, u_lid=tuple(cfg.u_lid), storage="f32", variant="aa",
                  lattice=q)
    lat.init_equilibrium()
    lat.step(20)
    f20 = gpu_state(lat)
    lat.step(1)
    f21 = gpu_state(lat)
    err_even = relmax(f21, oracle.run(cfg, f20, 1))
    del f20
    lat.step(1)
    err_odd = relmax(gpu_state(lat), oracle.run(cfg, f21, 1))
    print(f"D3Q{q} aa: full-lattice relative max error even {err_even:.3e} odd {err_odd:.3e}")
    assert err_even <= 1.5e-7 and err_odd <= 1.5e-7
