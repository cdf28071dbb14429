"""The C oracle against a separately written numpy collide-then-stream on
tiny grids (different lattice construction, whole-field passes, vector-keyed
directions)."""
import numpy as np
import pytest

import oracle
from oracle import BC_LID, BC_PERIODIC, BC_WALL, FORCE_FIELD, FORCE_UNIFORM, brute
from paper_2208_05429_gb300 import inputs
from helpers import noisy_equilibrium


def _to_brute(f_oracle):
    c_o, _, _ = oracle.lattice()
    c_b, _ = brute.velocity_set()
    idx = {tuple(v): k for k, v in enumerate(c_o)}
    return np.stack([f_oracle[idx[tuple(v)]] for v in c_b])


CASES = {
    "cavity": dict(nx=8, ny=8, nz=8, tau=0.6, bc=(BC_WALL,) * 5 + (BC_LID,), u_lid=(0.05, 0.0, 0.0)),
    "channel_force": dict(nx=8, ny=7, nz=6, tau=0.7, bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL, BC_WALL, BC_WALL),
                          force_mode=FORCE_UNIFORM, force_uniform=(1e-4, 0.0, 0.0)),
    "periodic_field": dict(nx=8, ny=8, nz=8, tau=0.55, force_mode=FORCE_FIELD),
    "mixed_lids": dict(nx=6, ny=8, nz=5, tau=0.9, bc=(BC_LID, BC_WALL, BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_LID),
                       u_lid=(0.0, 0.04, -0.01)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_equals_numpy_brute_force(name):
    kw = dict(CASES[name])
    cfg = oracle.Config(**kw)
    F = np.zeros((3, *cfg.shape))
    if cfg.force_mode == FORCE_FIELD:
        cfg.force_field = inputs.channel_force(cfg.nx, cfg.ny, cfg.nz, seed=5, sigma=1e-4).astype(np.float64)
        F = cfg.force_field
    elif cfg.force_mode == FORCE_UNIFORM:
        F[:] = np.array(cfg.force_uniform)[:, None, None, None]
    f = noisy_equilibrium(cfg, seed=hash(name) % 1000)
    fb = _to_brute(f)
    for _ in range(5):
        f = oracle.step(cfg, f)
        fb = brute.step(fb, cfg.tau, cfg.bc, cfg.u_lid, F, cfg.rho_wall)
    assert np.max(np.abs(_to_brute(f) - fb)) < 1e-14
