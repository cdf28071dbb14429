"""Second, separately written FP64 D3Q15 / D3Q19 / D3Q27 update in numpy (test
infrastructure).

This is a brute-force cross-check of ``lbm_oracle.c`` on tiny grids.  It is
written differently on purpose:

* the velocity set is generated (the vectors of {-1,0,1}^3 whose |c|^2 the
  lattice admits: {0,1,2} for D3Q19, {0,1,3} for D3Q15, all for D3Q27) and the
  weights come from |c|^2, instead of a typed-in table;
* collision runs on the whole field at once, then streaming moves each
  population plane with explicit target-index arithmetic, then the links that
  leave a non-periodic face are bounced back -- three separate passes, where the
  C oracle does collide-and-scatter cell by cell;
* populations are indexed by velocity vector, not by direction number, so the
  comparison with the C oracle goes through the vectors each side reports.

The update is the plain collide-then-stream of one time step (Fu & Song,
Sec. 3: collide, revert and swap_stream of a cell together amount to one
collision followed by streaming to the neighbours), with BGK + Guo forcing and
half-way bounce-back / moving lid as stated in the header of ``lbm_oracle.c``.
"""
from __future__ import annotations

import itertools

import numpy as np


# weight of a vector by its squared length, per lattice
WEIGHTS = {
    15: {0: 2.0 / 9.0, 1: 1.0 / 9.0, 3: 1.0 / 72.0},
    19: {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0},
    27: {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0},
}


def velocity_set(q=19):
    """D3Q<q> vectors and weights built from |c|^2 (order: sorted tuples)."""
    weight_of = WEIGHTS[q]
    cs = [c for c in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in c) in weight_of]
    cs.sort()
    c = np.array(cs, dtype=np.int64)
    w = np.array([weight_of[int((v * v).sum())] for v in c])
    assert len(c) == q
    return c, w


def collide(f, tau, F):
    """Post-collision populations for a whole field f[q, nz, ny, nx].
    F is [3, nz, ny, nx] (zeros for no force)."""
    c, w = velocity_set(f.shape[0])
    rho = f.sum(axis=0)
    mom = np.einsum("qa,qzyx->azyx", c.astype(np.float64), f)
    u = (mom + 0.5 * F) / rho
    cu = np.einsum("qa,azyx->qzyx", c.astype(np.float64), u)
    cF = np.einsum("qa,azyx->qzyx", c.astype(np.float64), F)
    usq = (u * u).sum(axis=0)
    uF = (u * F).sum(axis=0)
    wq = w[:, None, None, None]
    feq = wq * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
    S = wq * (3.0 * (cF - uF) + 9.0 * cu * cF)
    om = 1.0 / tau
    return f - om * (f - feq) + (1.0 - 0.5 * om) * S


def stream(fs, periodic, face_lid, u_lid, rho_wall=1.0):
    """Move post-collision populations to their targets.

    periodic: (px, py, pz) booleans; face_lid: dict face-> bool for the six
    faces (0:x-,1:x+,2:y-,3:y+,4:z-,5:z+)."""
    q, nz, ny, nx = fs.shape
    c, w = velocity_set(q)
    dims = (nx, ny, nz)
    out = np.full_like(fs, np.nan)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = (xx, yy, zz)
    index_of = {tuple(v): k for k, v in enumerate(c)}
    for i in range(q):
        tgt = []
        leaves = np.zeros((nz, ny, nx), bool)
        lid = np.zeros((nz, ny, nx), bool)
        for a in range(3):
            t = pos[a] + c[i, a]
            below, above = t < 0, t >= dims[a]
            if periodic[a]:
                t = np.mod(t, dims[a])
            else:
                leaves |= below | above
                lid |= (below & face_lid[2 * a]) | (above & face_lid[2 * a + 1])
            tgt.append(t)
        inside = ~leaves
        # links that stay in the box
        out[i, tgt[2][inside], tgt[1][inside], tgt[0][inside]] = fs[i][inside]
        # links that hit a wall come back into the opposite slot of the same cell
        o = index_of[tuple(-c[i])]
        cu_w = float(np.dot(c[i], u_lid))
        corr = np.where(lid, 6.0 * w[i] * rho_wall * cu_w, 0.0)
        out[o][leaves] = (fs[i] - corr)[leaves]
    assert not np.isnan(out).any(), "every slot must be written exactly once"
    return out


def step(f, tau, bc, u_lid=(0.0, 0.0, 0.0), F=None, rho_wall=1.0):
    """One collide-then-stream step of f[q, nz, ny, nx] (velocity_set order)."""
    if F is None:
        F = np.zeros((3,) + f.shape[1:])
    periodic = tuple(bc[2 * a] == 0 for a in range(3))
    face_lid = {k: bc[k] == 2 for k in range(6)}
    return stream(collide(f, tau, F), periodic, face_lid, np.asarray(u_lid, float), rho_wall)
