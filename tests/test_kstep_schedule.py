"""The K-step sweep's schedule (k_ksweep), restated on the host and checked
against the FP64 oracle.

The kernel's tile (16 x 8 for K = 3, 16 x 4 for K = 4), its levels s = 0 ..
K-1 of post-collision values on the tile widened by K - s cells, the rings
of three planes per level, the pipeline stage t = -K .. nz-1+K in which
level s produces plane t - s, the wrapped reads of periodic axes and the
half-way bounce-back with the lid term are written out below in plain numpy,
with every shared-memory index checked against its ring's bounds.  The K
steps it produces must equal K steps of the oracle exactly (the same
collision in FP64, the same additions): a wrong halo width, ring slot,
pipeline lag or wall test changes the result or trips a bound."""
import numpy as np
import pytest

import oracle
from helpers import noisy_equilibrium

C, W, OPP = oracle.lattice()
Q = 19
TILES = {3: (16, 8), 4: (16, 4)}


def _ksweep(cfg, f, K, TX, TY):
    n = (cfg.nx, cfg.ny, cfg.nz)
    per = [cfg.bc[2 * a] == oracle.BC_PERIODIC for a in range(3)]
    lidf = [cfg.bc[k] == oracle.BC_LID for k in range(6)]
    lid_term = [6.0 * W[i] * cfg.rho_wall * float(C[i] @ np.array(cfg.u_lid)) for i in range(Q)]
    out = np.full_like(f, np.nan)
    zero_force = np.zeros(3)
    for y0 in range(0, cfg.ny, TY):
        for x0 in range(0, cfg.nx, TX):
            halo = [K - s for s in range(K)] + [0]
            rw = [TX + 2 * h for h in halo]
            rh = [TY + 2 * h for h in halo]
            ring = [np.full((3, Q, rh[s], rw[s]), np.nan) for s in range(K)]

            def live(p, s):
                if s == K:
                    return 0 <= p < cfg.nz
                return 0 <= p < cfg.nz or (per[2] and -halo[s] <= p < cfg.nz + halo[s])

            for t in range(-K, cfg.nz + K):
                for s in range(K + 1):
                    p = t - s
                    if not live(p, s):
                        continue
                    h = halo[s]
                    for ry in range(rh[s]):
                        for rx in range(rw[s]):
                            X, Y = x0 - h + rx, y0 - h + ry
                            if (not per[0] and not 0 <= X < n[0]) or (not per[1] and not 0 <= Y < n[1]):
                                continue
                            wx, wy, wz = X % n[0], Y % n[1], p % n[2]
                            if s == 0:
                                v = f[:, wz, wy, wx].copy()
                            else:
                                v = np.empty(Q)
                                lv = ring[s - 1]
                                for i in range(Q):
                                    src = (X - C[i][0], Y - C[i][1], p - C[i][2])
                                    wall, lid = False, False
                                    for a in range(3):
                                        if not per[a] and not 0 <= src[a] < n[a]:
                                            wall = True
                                            lid |= lidf[2 * a + (0 if src[a] < 0 else 1)]
                                    if wall:
                                        qx, qy = rx + 1, ry + 1
                                        assert 0 <= qx < rw[s - 1] and 0 <= qy < rh[s - 1]
                                        v[i] = lv[p % 3, OPP[i], qy, qx] + (lid_term[i] if lid else 0.0)
                                    else:
                                        assert live(src[2], s - 1)
                                        qx, qy = rx + 1 - C[i][0], ry + 1 - C[i][1]
                                        assert 0 <= qx < rw[s - 1] and 0 <= qy < rh[s - 1]
                                        v[i] = lv[src[2] % 3, i, qy, qx]
                                    assert np.isfinite(v[i]), "read of a value no level produced"
                            if s == K:
                                if X < n[0] and Y < n[1]:
                                    out[:, wz, wy, wx] = v
                            else:
                                ring[s][p % 3, :, ry, rx] = oracle.collide_cell(cfg.tau, v, zero_force)
    return out


CASES = {
    "cavity_20x11x6": oracle.cavity(20, 0.6, ny=11, nz=6),
    "channel_18x9x5": oracle.Config(nx=18, ny=9, nz=5, tau=0.7, bc=(0, 0, 1, 1, 1, 1)),
    "periodic_5x3x4": oracle.Config(nx=5, ny=3, nz=4, tau=0.8),
    "lids_17x5x3": oracle.Config(nx=17, ny=5, nz=3, tau=0.9, bc=(2, 1, 0, 0, 1, 2), u_lid=(0.0, 0.04, -0.01)),
    "pencil_1x2x3": oracle.Config(nx=1, ny=2, nz=3, tau=0.75, bc=(0, 0, 1, 2, 0, 0), u_lid=(0.02, 0.0, 0.0)),
}


@pytest.mark.parametrize("K", [3, 4])
@pytest.mark.parametrize("name", sorted(CASES))
def test_schedule_equals_k_oracle_steps(K, name):
    cfg = CASES[name]
    f = noisy_equilibrium(cfg, seed=K)
    got = _ksweep(cfg, f, K, *TILES[K])
    assert not np.isnan(got).any(), "every cell written once"
    assert np.array_equal(got, oracle.run(cfg, f, K))


def test_shared_memory_fits():
    """Rings of the kernel's tiles: 3 planes x 19 directions x FP32 per level."""
    for K, (TX, TY) in TILES.items():
        cells = sum((TX + 2 * (K - s)) * (TY + 2 * (K - s)) for s in range(K))
        assert 3 * Q * 4 * cells <= 227 * 1024, K
