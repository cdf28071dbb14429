"""The paper's own CPU algorithms for the D3Q19 update, as a timed host
comparator (Fu & Song, arXiv 2208.05429): the fused swap LBM (Sec. 3,
Alg. 1), the sequential two-step memory-aware LBM with prism traversal
(Sec. 4.1, Alg. 2) and its OpenMP form with intersection layers (Sec. 4.2,
Alg. 3).  The arithmetic is in ``lbm_memaware.c`` (double precision, compiled
without floating-point contraction); this module compiles it on first use
and marshals numpy arrays through ctypes.

Two builds: the timed one, and one with the dependency checker
(``-DMEM_CHECK``) that counts every collision or link exchange made out of
the order the swap scheme allows (``checked=True`` below).

Arrays: ``f[19, nz, ny, nx]`` in this library's direction order
(:func:`lattice`); internally the populations are stored cell by cell,
``[nz, ny, nx, 19]``, as the paper's solvers store them.  Faces are walls
(1) or lids (2) in the order x-, x+, y-, y+, z-, z+; periodic faces are
rejected.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

Q = 19
WALL, LID = 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_memaware.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {False: os.path.join(_BUILD, "liblbm_memaware.so"), True: os.path.join(_BUILD, "liblbm_memaware_check.so")}
_lock = threading.Lock()
_loaded = {}


def build(force: bool = False) -> None:
    """Compile the timed and the checked library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    for checked, path in _LIBS.items():
        if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
            continue
        tmp = path + f".{os.getpid()}.tmp"
        flags = ["-O1", "-DMEM_CHECK"] if checked else ["-O3"]
        cmd = ["gcc", *flags, "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", _SRC, "-o", tmp,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("bc", ctypes.c_int32 * 6),
        ("u_lid", ctypes.c_double * 3),
        ("rho_wall", ctypes.c_double),
        ("force_mode", ctypes.c_int32),
        ("force_uniform", ctypes.c_double * 3),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _lib(checked: bool):
    with _lock:
        if checked not in _loaded:
            build()
            lib = ctypes.CDLL(_LIBS[checked])
            P = ctypes.POINTER(_Cfg)
            lib.mem_fuse.argtypes = [P, _D, ctypes.c_int64]
            lib.mem_two_step_prism.argtypes = [P, _D, ctypes.c_int64, ctypes.c_int64]
            lib.mem_two_step_prism_omp.argtypes = [P, _D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
            lib.mem_lattice.argtypes = [ctypes.POINTER(ctypes.c_int32), _D]
            lib.mem_check_violations.restype = ctypes.c_int64
            lib.mem_checked.restype = ctypes.c_int
            if checked:
                lib.mem_check_planted_misorder.argtypes = [P, _D]
                lib.mem_check_planted_misorder.restype = ctypes.c_int64
            _loaded[checked] = lib
        return _loaded[checked]


@dataclass
class Config:
    nx: int
    ny: int
    nz: int
    tau: float
    bc: Sequence[int] = (WALL, WALL, WALL, WALL, WALL, LID)
    u_lid: Sequence[float] = (0.05, 0.0, 0.0)
    rho_wall: float = 1.0
    force_uniform: Optional[Sequence[float]] = None

    def c_struct(self) -> _Cfg:
        c = _Cfg()
        c.nx, c.ny, c.nz, c.tau = int(self.nx), int(self.ny), int(self.nz), float(self.tau)
        for k in range(6):
            c.bc[k] = int(self.bc[k])
        for a in range(3):
            c.u_lid[a] = float(self.u_lid[a])
        c.rho_wall = float(self.rho_wall)
        c.force_mode = 0 if self.force_uniform is None else 1
        for a in range(3):
            c.force_uniform[a] = 0.0 if self.force_uniform is None else float(self.force_uniform[a])
        return c

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.nz, self.ny, self.nx)


def lattice() -> Tuple[np.ndarray, np.ndarray]:
    """(c[19, 3] as (c_x, c_y, c_z), w[19]) in this library's direction order."""
    c = (ctypes.c_int32 * (3 * Q))()
    w = (ctypes.c_double * Q)()
    _lib(False).mem_lattice(c, w)
    return np.array(c, dtype=np.int64).reshape(Q, 3), np.array(w)


def to_cells(f: np.ndarray) -> np.ndarray:
    """[19, nz, ny, nx] -> the cell-by-cell layout [nz, ny, nx, 19] (a copy)."""
    return np.ascontiguousarray(np.moveaxis(np.asarray(f, dtype=np.float64), 0, -1))


def from_cells(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(a, -1, 0))


def _check(rc: int, name: str) -> None:
    if rc != 0:
        raise ValueError(f"{name}: status {rc}")


def run_cells(alg: str, cfg: Config, cells: np.ndarray, nsteps: int, tile: int = 0, nthreads: int = 0,
              checked: bool = False) -> None:
    """Step the cell-by-cell array in place: alg = "fuse" (Alg. 1), "two_step"
    (Alg. 2, prism stride `tile`, 0 = no prisms) or "omp" (Alg. 3 on
    `nthreads` threads, 0 = all)."""
    assert cells.dtype == np.float64 and cells.flags.c_contiguous and cells.shape == (*cfg.shape, Q)
    lib = _lib(checked)
    c = cfg.c_struct()
    p = cells.ctypes.data_as(_D)
    if alg == "fuse":
        _check(lib.mem_fuse(ctypes.byref(c), p, int(nsteps)), alg)
    elif alg == "two_step":
        _check(lib.mem_two_step_prism(ctypes.byref(c), p, int(nsteps), int(tile)), alg)
    elif alg == "omp":
        _check(lib.mem_two_step_prism_omp(ctypes.byref(c), p, int(nsteps), int(tile), int(nthreads)), alg)
    else:
        raise ValueError(alg)


def run(alg: str, cfg: Config, f: np.ndarray, nsteps: int, tile: int = 0, nthreads: int = 0,
        checked: bool = False) -> np.ndarray:
    """As run_cells, on f[19, nz, ny, nx]; returns the new populations."""
    cells = to_cells(f)
    run_cells(alg, cfg, cells, nsteps, tile, nthreads, checked)
    return from_cells(cells)


def violations() -> int:
    """Order violations the checker has counted since reset_violations()."""
    return int(_lib(True).mem_check_violations())


def reset_violations() -> None:
    _lib(True).mem_check_reset()


def planted_misorder(cfg: Config, f: np.ndarray) -> int:
    """Checker self-test: one step of Alg. 1 with Stage II before Stage I;
    returns the violations the checker counted (expected > 0)."""
    cells = to_cells(f)
    c = cfg.c_struct()
    return int(_lib(True).mem_check_planted_misorder(ctypes.byref(c), cells.ctypes.data_as(_D)))
