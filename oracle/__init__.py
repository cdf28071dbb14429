"""Test-only FP64 oracle of the D3Q19 (also D3Q15, D3Q27) BGK collide-and-stream update.

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` import it; the product package never
does, and the two share no code.  The arithmetic lives in ``lbm_oracle.c``
(plain C, double precision, compiled without floating-point contraction so that
x86 and Arm hosts give the same bits); this module only compiles it on first
use and marshals numpy arrays through ctypes.

Arrays use the canonical layout: populations ``f[q, nz, ny, nx]`` (q = 19, or
``Config.q`` = 15 or 27) in the
oracle's own direction order (see :func:`lattice`), densities ``rho[nz, ny, nx]``
and velocities ``u[3, nz, ny, nx]``.

What the functions compute is stated in the header of ``lbm_oracle.c``: the
D3Q19 lattice with directions 1..9 forming the swap half of Sec. 3 of Fu & Song
(arXiv 2208.05429) and i+9 their opposites, BGK collision with Guo forcing,
periodic or half-way bounce-back faces with a moving lid, and the discrete
adjoint of that step.  Every function is pinned by the CPU tests
(``tests/test_oracle_*.py``) against lattice identities, closed-form flows,
conservation laws, a separately written numpy collide-then-stream and finite
differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

Q = 19
LATTICES = (15, 19, 27)
BC_PERIODIC, BC_WALL, BC_LID = 0, 1, 2
FORCE_NONE, FORCE_UNIFORM, FORCE_FIELD = 0, 1, 2
COLL_BGK, COLL_TRT, COLL_REG, COLL_MRT = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("bc", ctypes.c_int32 * 6),
        ("u_lid", ctypes.c_double * 3),
        ("rho_wall", ctypes.c_double),
        ("force_mode", ctypes.c_int32),
        ("force_uniform", ctypes.c_double * 3),
        ("force_field", ctypes.POINTER(ctypes.c_double)),
        ("collision", ctypes.c_int32),
        ("trt_lambda", ctypes.c_double),
        ("mrt_s3", ctypes.c_double),
        ("mrt_s4", ctypes.c_double),
        ("q", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Cfg)
            sigs = {
                "orc_lattice": [_I32, _D, _I32],
                "orc_lattice_q": [ctypes.c_int32, _I32, _D, _I32],
                "orc_equilibrium": [ctypes.c_double, _D, _D],
                "orc_equilibrium_q": [ctypes.c_int32, ctypes.c_double, _D, _D],
                "orc_collide_cell_q": [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _D, _D, _D],
                "orc_collide_cell": [ctypes.c_double, _D, _D, _D],
                "orc_collide_cell_trt": [ctypes.c_double, ctypes.c_double, _D, _D, _D],
                "orc_collide_cell_reg": [ctypes.c_double, _D, _D, _D],
                "orc_collide_cell_mrt": [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D, _D],
                "orc_init_equilibrium": [P, _D, _D, _D],
                "orc_step": [P, _D, _D],
                "orc_run": [P, _D, ctypes.c_int64, _D],
                "orc_step_cells": [P, _D, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _D],
                "orc_moments": [P, _D, _D, _D],
                "orc_reduce": [P, _D, _D],
                "orc_adjoint_step": [P, _D, _D, _D, _D],
                "orc_adjoint_seed": [P, _D, _D, _D, _D, _D],
            }
            for name, argt in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = None
            lib.orc_threads.argtypes = [ctypes.c_int]
            lib.orc_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous float64"
    return a.ctypes.data_as(_D)


@dataclass
class Config:
    """Problem definition shared by every oracle call.

    ``bc`` lists the faces x-, x+, y-, y+, z-, z+ (BC_PERIODIC, BC_WALL, BC_LID);
    ``force_field`` is a float64 array [3, nz, ny, nx] used when
    ``force_mode == FORCE_FIELD``.
    """
    nx: int
    ny: int
    nz: int
    tau: float
    bc: Sequence[int] = (BC_PERIODIC,) * 6
    u_lid: Sequence[float] = (0.0, 0.0, 0.0)
    rho_wall: float = 1.0
    force_mode: int = FORCE_NONE
    force_uniform: Sequence[float] = (0.0, 0.0, 0.0)
    force_field: Optional[np.ndarray] = field(default=None, repr=False)
    collision: int = 0            # COLL_BGK, COLL_TRT, COLL_REG or COLL_MRT
    trt_lambda: float = 3.0 / 16.0
    mrt_s3: float = 1.0           # MRT rates of the third- and fourth-order moments
    mrt_s4: float = 1.0
    q: int = 19                   # lattice: D3Q15, D3Q19 or D3Q27 (MRT: D3Q19 only)

    def __post_init__(self):
        if self.q not in LATTICES:
            raise ValueError(f"lattice q={self.q}: one of {LATTICES}")
        if self.q != 19 and self.collision == COLL_MRT:
            raise ValueError("the MRT collision is defined on D3Q19 only")

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def _c(self) -> _Cfg:
        c = _Cfg()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.tau = float(self.tau)
        for k in range(6):
            c.bc[k] = int(self.bc[k])
        for a in range(3):
            c.u_lid[a] = float(self.u_lid[a])
            c.force_uniform[a] = float(self.force_uniform[a])
        c.rho_wall = float(self.rho_wall)
        c.force_mode = int(self.force_mode)
        c.collision = int(self.collision)
        c.trt_lambda = float(self.trt_lambda)
        c.mrt_s3 = float(self.mrt_s3)
        c.mrt_s4 = float(self.mrt_s4)
        c.q = int(self.q)
        if self.force_mode == FORCE_FIELD:
            ff = np.ascontiguousarray(self.force_field, dtype=np.float64).reshape(3, *self.shape)
            self._ff_keep = ff  # keep the buffer alive for the call
            c.force_field = _ptr(ff)
        else:
            c.force_field = None
        return c


def cavity(n: int, tau: float, u_lid=(0.05, 0.0, 0.0), ny: int = None, nz: int = None) -> Config:
    """Lid-driven cavity: lid on the z+ face, half-way bounce-back elsewhere."""
    return Config(nx=n, ny=ny or n, nz=nz or n, tau=tau,
                  bc=(BC_WALL, BC_WALL, BC_WALL, BC_WALL, BC_WALL, BC_LID), u_lid=u_lid)


def lattice(q: int = 19):
    """The oracle's own table of lattice D3Q<q>: (c[q,3] int, w[q], opp[q] int)."""
    lib = _load()
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    opp = np.zeros(q, np.int32)
    if q == 19:
        lib.orc_lattice(c.ctypes.data_as(_I32), _ptr(w), opp.ctypes.data_as(_I32))
    else:
        assert q in LATTICES, q
        lib.orc_lattice_q(q, c.ctypes.data_as(_I32), _ptr(w), opp.ctypes.data_as(_I32))
    return c.astype(np.int64), w, opp.astype(np.int64)


def equilibrium(rho: float, u, q: int = 19) -> np.ndarray:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(q, np.float64)
    if q == 19:
        lib.orc_equilibrium(float(rho), _ptr(uu), _ptr(out))
    else:
        assert q in LATTICES, q
        lib.orc_equilibrium_q(q, float(rho), _ptr(uu), _ptr(out))
    return out


def collide_cell_q(q: int, tau: float, f, F=(0.0, 0.0, 0.0), collision: int = COLL_BGK,
                   lam: float = 3.0 / 16.0) -> np.ndarray:
    """One cell of lattice D3Q<q>: BGK, TRT (Lambda = lam) or regularised BGK."""
    assert q in LATTICES and collision in (COLL_BGK, COLL_TRT, COLL_REG)
    lib = _load()
    ff = np.ascontiguousarray(f, dtype=np.float64)
    assert ff.shape == (q,)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(q, np.float64)
    lib.orc_collide_cell_q(int(q), int(collision), float(tau), float(lam), _ptr(ff), _ptr(FF), _ptr(out))
    return out


def collide_cell_mrt(tau: float, s3: float, s4: float, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    lib = _load()
    ff = np.ascontiguousarray(f, dtype=np.float64)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q, np.float64)
    lib.orc_collide_cell_mrt(float(tau), float(s3), float(s4), _ptr(ff), _ptr(FF), _ptr(out))
    return out


def collide_cell_reg(tau: float, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    lib = _load()
    ff = np.ascontiguousarray(f, dtype=np.float64)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q, np.float64)
    lib.orc_collide_cell_reg(float(tau), _ptr(ff), _ptr(FF), _ptr(out))
    return out


def collide_cell_trt(tau: float, lam: float, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    lib = _load()
    ff = np.ascontiguousarray(f, dtype=np.float64)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q, np.float64)
    lib.orc_collide_cell_trt(float(tau), float(lam), _ptr(ff), _ptr(FF), _ptr(out))
    return out


def collide_cell(tau: float, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
    lib = _load()
    ff = np.ascontiguousarray(f, dtype=np.float64)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q, np.float64)
    lib.orc_collide_cell(float(tau), _ptr(ff), _ptr(FF), _ptr(out))
    return out


def store_round(f: np.ndarray, storage: str) -> np.ndarray:
    """The populations f[q, ...] (q = 15, 19 or 27) as a 16-bit shifted storage format holds
    them: s_i = f_i - w_i rounded to nearest-even, "f16s" to IEEE binary16,
    "bf16s" to bfloat16 (of s_i rounded to binary32 first, the compute type
    that produces it), and returned as w_i + s_i in float64; also the stored
    s itself.  Plain numpy; the definition of the storage, not of the step."""
    _, w, _ = lattice(np.shape(f)[0])
    shp = (-1,) + (1,) * (np.ndim(f) - 1)
    s = np.asarray(f, dtype=np.float64) - w.reshape(shp)
    if storage == "f16s":
        r = s.astype(np.float16).astype(np.float64)
    elif storage == "bf16s":
        x = s.astype(np.float32).view(np.uint32).astype(np.uint64)
        x = (x + 0x7FFF + ((x >> 16) & 1)) & 0xFFFF0000
        r = x.astype(np.uint32).view(np.float32).astype(np.float64)
    else:
        raise ValueError(storage)
    return r + w.reshape(shp), r


def init_equilibrium(cfg: Config, rho=None, u=None) -> np.ndarray:
    lib = _load()
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(cfg.shape)
    v = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(3, *cfg.shape)
    f = np.zeros((cfg.q, *cfg.shape), np.float64)
    lib.orc_init_equilibrium(ctypes.byref(cfg._c()), _ptr(r), _ptr(v), _ptr(f))
    return f


def step(cfg: Config, f: np.ndarray) -> np.ndarray:
    lib = _load()
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(fin)
    lib.orc_step(ctypes.byref(cfg._c()), _ptr(fin), _ptr(out))
    return out


def step_cells(cfg: Config, f: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """f^{t+1}[k, 19] at the cells [k, 3] = (x, y, z) only, from the state f."""
    lib = _load()
    fin = np.ascontiguousarray(f, dtype=np.float64)
    xyz = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(xyz), cfg.q), np.float64)
    lib.orc_step_cells(ctypes.byref(cfg._c()), _ptr(fin), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                       len(xyz), _ptr(out))
    return out


def threads(n: int = 0) -> int:
    """OpenMP threads of the oracle from now on (n >= 1), or just the number in
    effect (n = 0).  For host timing only: results do not depend on it."""
    return int(_load().orc_threads(int(n)))


def run(cfg: Config, f: np.ndarray, nsteps: int) -> np.ndarray:
    lib = _load()
    cur = np.array(f, dtype=np.float64, order="C", copy=True)
    tmp = np.empty_like(cur)
    lib.orc_run(ctypes.byref(cfg._c()), _ptr(cur), int(nsteps), _ptr(tmp))
    return cur


def moments(cfg: Config, f: np.ndarray):
    lib = _load()
    fin = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.empty(cfg.shape, np.float64)
    u = np.empty((3, *cfg.shape), np.float64)
    lib.orc_moments(ctypes.byref(cfg._c()), _ptr(fin), _ptr(rho), _ptr(u))
    return rho, u


def reduce(cfg: Config, f: np.ndarray) -> np.ndarray:
    """[mass, momentum_x, momentum_y, momentum_z, kinetic energy] in FP64."""
    lib = _load()
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(5, np.float64)
    lib.orc_reduce(ctypes.byref(cfg._c()), _ptr(fin), _ptr(out))
    return out


def adjoint_step(cfg: Config, f_t: np.ndarray, lam_next: np.ndarray, gF: np.ndarray) -> np.ndarray:
    """lam_t = (d f^{t+1} / d f^t)^T lam_next; gF[3, ...] += (d f^{t+1} / d F)^T lam_next."""
    lib = _load()
    ft = np.ascontiguousarray(f_t, dtype=np.float64)
    ln = np.ascontiguousarray(lam_next, dtype=np.float64)
    assert gF.dtype == np.float64 and gF.flags["C_CONTIGUOUS"]
    out = np.empty_like(ft)
    lib.orc_adjoint_step(ctypes.byref(cfg._c()), _ptr(ft), _ptr(ln), _ptr(out), _ptr(gF))
    return out


def adjoint_seed(cfg: Config, f: np.ndarray, dLdrho, dLdu, gF: np.ndarray) -> np.ndarray:
    """dL/df for a loss of the output moments (rho, u) of state f; adds the
    half-force path of u into gF."""
    lib = _load()
    fin = np.ascontiguousarray(f, dtype=np.float64)
    dr = None if dLdrho is None else np.ascontiguousarray(dLdrho, dtype=np.float64).reshape(cfg.shape)
    du = np.ascontiguousarray(dLdu, dtype=np.float64).reshape(3, *cfg.shape)
    lam = np.empty_like(fin)
    lib.orc_adjoint_seed(ctypes.byref(cfg._c()), _ptr(fin), _ptr(dr), _ptr(du), _ptr(lam), _ptr(gF))
    return lam


def forward_with_states(cfg: Config, f0: np.ndarray, nsteps: int):
    """All states f^0..f^T of a forward run (small grids only)."""
    states = [np.array(f0, dtype=np.float64, copy=True)]
    for _ in range(nsteps):
        states.append(step(cfg, states[-1]))
    return states


def adjoint_run(cfg: Config, f0: np.ndarray, nsteps: int, dLdu_fn, dLdrho_fn=None):
    """Reverse sweep over nsteps for a loss L(rho^T, u^T).

    ``dLdu_fn(rho, u)`` returns dL/du [3, ...] at the final state (and
    ``dLdrho_fn`` dL/drho, optional).  Returns (dL/df^0, dL/dF per cell)."""
    states = forward_with_states(cfg, f0, nsteps)
    rho, u = moments(cfg, states[-1])
    gF = np.zeros((3, *cfg.shape), np.float64)
    lam = adjoint_seed(cfg, states[-1], None if dLdrho_fn is None else dLdrho_fn(rho, u),
                       dLdu_fn(rho, u), gF)
    for t in range(nsteps - 1, -1, -1):
        lam = adjoint_step(cfg, states[t], lam, gF)
    return lam, gF
