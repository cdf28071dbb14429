"""Shared GPU-test plumbing: the synthetic cases, construction of a GPU
lattice matching an oracle configuration, and population conversions
between the two direction numberings."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import BC_LID, BC_PERIODIC, BC_WALL, FORCE_FIELD, FORCE_NONE, FORCE_UNIFORM
from paper_2208_05429_gb300 import inputs
from paper_2208_05429_gb300.lbm import Lattice, lbm_lattice, lbm_lattice_q
from helpers import noisy_equilibrium, perm_oracle_to

P, W, L = BC_PERIODIC, BC_WALL, BC_LID


def cases():
    """name -> oracle.Config; sizes are ragged against the 32 x {4,8,16}
    tiles, include single-cell-wide tiles, periodic wraps on every axis,
    lids on several faces and all three force modes."""
    c = {}
    c["cavity16"] = oracle.cavity(16, 0.6)
    c["channel_37x19x23"] = oracle.Config(nx=37, ny=19, nz=23, tau=0.7, bc=(P, P, W, W, W, W),
                                          force_mode=FORCE_UNIFORM, force_uniform=(1e-5, 0.0, 2e-6))
    pf = oracle.Config(nx=20, ny=18, nz=17, tau=0.55, force_mode=FORCE_FIELD)
    pf.force_field = inputs.channel_force(20, 18, 17, seed=77, sigma=1e-5).astype(np.float64)
    c["periodic_field_20x18x17"] = pf
    c["mixed_33x40x9"] = oracle.Config(nx=33, ny=40, nz=9, tau=0.9, bc=(L, W, P, P, W, L), u_lid=(0.0, 0.04, -0.01))
    c["flat_40x35x1"] = oracle.Config(nx=40, ny=35, nz=1, tau=0.65, bc=(W, W, W, L, P, P), u_lid=(0.03, 0.0, 0.0))
    c["line_70x1x1"] = oracle.Config(nx=70, ny=1, nz=1, tau=0.8)
    c["periodic_33x15x2"] = oracle.Config(nx=33, ny=15, nz=2, tau=0.7, force_mode=FORCE_UNIFORM,
                                          force_uniform=(0.0, 3e-6, -2e-6))
    # rows made only of x-edge cells (nx = 2, nx = 1)
    c["narrow_2x21x5"] = oracle.Config(nx=2, ny=21, nz=5, tau=0.75, bc=(W, L, P, P, W, W), u_lid=(0.0, 0.02, 0.01))
    c["pencil_1x19x4"] = oracle.Config(nx=1, ny=19, nz=4, tau=0.8, bc=(P, P, W, L, W, W), u_lid=(0.02, 0.0, 0.0))
    return c


def gpu_perm(q: int = 19):
    c_gpu, _ = lbm_lattice() if q == 19 else lbm_lattice_q(q)
    p = perm_oracle_to(c_gpu)          # c_gpu[p[k]] == c_oracle[k]
    inv = np.empty_like(p)
    inv[p] = np.arange(len(p))
    return p, inv


def to_gpu_order(f_oracle: np.ndarray) -> np.ndarray:
    _, inv = gpu_perm(len(f_oracle))
    return f_oracle[inv]


def to_oracle_order(f_gpu: np.ndarray) -> np.ndarray:
    p, _ = gpu_perm(len(f_gpu))
    return f_gpu[p]


def make_gpu(cfg: "oracle.Config", storage: str, variant: str, device="cuda:0") -> Lattice:
    import torch
    if cfg.force_mode == FORCE_FIELD:
        force = torch.tensor(np.asarray(cfg.force_field, dtype=np.float32), device=device)
    elif cfg.force_mode == FORCE_UNIFORM:
        force = tuple(cfg.force_uniform)
    else:
        force = None
    return Lattice((cfg.nx, cfg.ny, cfg.nz), cfg.tau, bc=tuple(int(b) for b in cfg.bc), u_lid=tuple(cfg.u_lid),
                   rho_wall=cfg.rho_wall, storage=storage, variant=variant, force=force, device=device,
                   collision={oracle.COLL_TRT: "trt", oracle.COLL_REG: "reg", oracle.COLL_MRT: "mrt"}.get(
                       cfg.collision, "bgk"),
                   trt_lambda=cfg.trt_lambda, mrt_s3=cfg.mrt_s3, mrt_s4=cfg.mrt_s4, lattice=cfg.q)


def oracle_force_as_f32(cfg: "oracle.Config") -> "oracle.Config":
    """The oracle sees exactly the FP32 force field the GPU reads."""
    if cfg.force_mode == FORCE_FIELD:
        cfg.force_field = np.asarray(cfg.force_field, dtype=np.float32).astype(np.float64)
    return cfg


def start_state(cfg: "oracle.Config", seed: int = 1) -> np.ndarray:
    """A seeded non-equilibrium state in oracle order (FP64)."""
    return noisy_equilibrium(cfg, seed=seed, amp=0.02, drho=0.01, umax=0.03)


def load_state(lat: Lattice, f_oracle: np.ndarray):
    import torch
    lat.init_populations(torch.tensor(to_gpu_order(f_oracle), dtype=torch.float64, device=lat.device))


def gpu_state(lat: Lattice) -> np.ndarray:
    import torch
    return to_oracle_order(lat.populations(torch.float64).cpu().numpy())


def gpu_moments(lat: Lattice):
    import torch
    rho, u = lat.moments(torch.float64)
    return rho.cpu().numpy(), u.cpu().numpy()
