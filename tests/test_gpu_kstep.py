"""The K-step sweep (KSTEP, K = 3 and 4 time steps per sweep on two
lattices) on the GPU, through the C ABI.

It reads every pulled value through the storage format, as the two-lattice
step stores and reloads it, and collides with the same function, so it must
equal K two-lattice steps bit for bit: on ragged shapes against its 16 x 8
and 16 x 4 tiles, periodic axes narrower than its halos, walls and lids on
several faces, uniform and per-cell force, every FP32-compute storage format,
step counts that leave a two-lattice remainder, and the whole 256^3 cavity.
Against the FP64 oracle: 1e-5 in u after 99 steps of the 32^3 cavity, and on
the whole 256^3 lattice one sweep from the GPU's own state within the FP32
bound of the other full-lattice checks (1.5e-7 per two steps: 2.5e-7 for 3)."""
import numpy as np
import pytest

import oracle
from gpu_cases import cases, gpu_moments, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state
from helpers import relmax

pytestmark = pytest.mark.gpu

NAMES = ["cavity16", "channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "flat_40x35x1",
         "line_70x1x1", "periodic_33x15x2", "narrow_2x21x5", "pencil_1x19x4"]


def _kstep(cfg, storage, K):
    import torch
    from paper_2208_05429_gb300.lbm import Lattice
    from oracle import FORCE_FIELD, FORCE_UNIFORM
    if cfg.force_mode == FORCE_FIELD:
        force = torch.tensor(np.asarray(cfg.force_field, dtype=np.float32), device="cuda:0")
    elif cfg.force_mode == FORCE_UNIFORM:
        force = tuple(cfg.force_uniform)
    else:
        force = None
    return Lattice((cfg.nx, cfg.ny, cfg.nz), cfg.tau, bc=tuple(int(b) for b in cfg.bc), u_lid=tuple(cfg.u_lid),
                   rho_wall=cfg.rho_wall, storage=storage, variant="kstep", force=force, device="cuda:0",
                   sweep_steps=K)


@pytest.mark.parametrize("K", [3, 4])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_equals_two_lattice(gpu, K, name, storage):
    import torch
    cfg = oracle_force_as_f32(cases()[name])
    f0 = start_state(cfg, seed=K)
    ks = _kstep(cfg, storage, K)
    load_state(ks, f0)
    tl = make_gpu(cfg, storage, "two_lattice")
    load_state(tl, f0)
    for n in (K, 2 * K + 1):
        ks.profile(True)
        ks.step(n)
        ran = ks.profile_read()
        ks.profile(False)
        tl.step(n)
        assert ran["kstep"][0] == n // K, ran
        assert torch.equal(ks.populations(torch.float64), tl.populations(torch.float64)), (name, n)
    assert ks.time == tl.time == 3 * K + 1


@pytest.mark.parametrize("storage", ["f32s", "bf16s"])
@pytest.mark.parametrize("name", ["cavity16", "periodic_field_20x18x17", "mixed_33x40x9"])
def test_other_formats_equal_two_lattice(gpu, storage, name):
    import torch
    cfg = oracle_force_as_f32(cases()[name])
    f0 = start_state(cfg, seed=11)
    ks = _kstep(cfg, storage, 3)
    load_state(ks, f0)
    tl = make_gpu(cfg, storage, "two_lattice")
    load_state(tl, f0)
    ks.step(40)           # graph replay: 13 sweeps and one two-lattice step per 40
    tl.step(40)
    assert torch.equal(ks.populations(torch.float64), tl.populations(torch.float64))


@pytest.mark.parametrize("K", [3, 4])
def test_cavity_32_fp32_99_steps(gpu, K):
    cfg = oracle.cavity(32, 0.6)
    ref = oracle.run(cfg, oracle.init_equilibrium(cfg), 99)
    _, u_r = oracle.moments(cfg, ref)
    lat = _kstep(cfg, "f32", K)
    lat.init_equilibrium()
    lat.step(99)
    _, u = gpu_moments(lat)
    assert relmax(u, u_r) <= 1e-5


@pytest.mark.parametrize("K", [3, 4])
def test_full_lattice_at_bench_size(gpu, K):
    """256^3 cavity, tau = 0.55, FP32: after 24 steps, one sweep against the
    FP64 oracle stepping the GPU's own state K times, and bit for bit against
    the two-lattice schedule from the same state."""
    import torch
    from paper_2208_05429_gb300.lbm import CAVITY_BC, Lattice
    cfg = oracle.cavity(256, 0.55)
    lat = Lattice((256, 256, 256), 0.55, bc=CAVITY_BC, u_lid=tuple(cfg.u_lid), storage="f32", variant="kstep",
                  sweep_steps=K)
    lat.init_equilibrium()
    lat.step(24)
    f24 = lat.populations(torch.float32)
    tl = Lattice((256, 256, 256), 0.55, bc=CAVITY_BC, u_lid=tuple(cfg.u_lid), storage="f32", variant="two_lattice")
    tl.init_populations(f24)
    tl.step(K)
    lat.step(K)
    assert torch.equal(lat.populations(torch.float32), tl.populations(torch.float32))
    del tl
    from gpu_cases import to_oracle_order
    f = to_oracle_order(f24.double().cpu().numpy())
    del f24
    err = relmax(gpu_state(lat), oracle.run(cfg, f, K))
    print(f"kstep K={K}: full-lattice relative max error after one sweep {err:.3e}")
    assert err <= 1.5e-7 * K / 2 + 1e-8
