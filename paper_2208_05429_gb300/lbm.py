"""ctypes binding of the C ABI in ``include/lbm.h``.

The module-level functions carry the C names (``lbm_create``,
``lbm_step``, ...) and only marshal arguments; every step of the lattice
update runs in the CUDA library ``_build/liblbm_gb300.so``.  PyTorch supplies
device memory (tensors' ``data_ptr()``) and streams.  There is no CPU
fallback: if the library is missing, loading it raises.

:class:`Lattice` wraps a handle for convenient use from Python.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional, Sequence, Tuple, Union

import numpy as np

Q = 19

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ESTATE, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_LID = 0, 1, 2
LBM_STORAGE_F64, LBM_STORAGE_F32, LBM_STORAGE_F32S, LBM_STORAGE_F16S, LBM_STORAGE_BF16S = 0, 1, 2, 3, 4
LBM_VARIANT_TWO_LATTICE, LBM_VARIANT_AA, LBM_VARIANT_MERGED, LBM_VARIANT_KSTEP = 0, 1, 2, 3
LBM_FORCE_NONE, LBM_FORCE_UNIFORM, LBM_FORCE_FIELD = 0, 1, 2
LBM_DTYPE_F32, LBM_DTYPE_F64 = 0, 1
LBM_LATTICE_D3Q15, LBM_LATTICE_D3Q19, LBM_LATTICE_D3Q27 = 15, 19, 27
LBM_COLLISION_BGK, LBM_COLLISION_TRT, LBM_COLLISION_REG, LBM_COLLISION_MRT = 0, 1, 2, 3
COLLISION = {"bgk": LBM_COLLISION_BGK, "trt": LBM_COLLISION_TRT, "reg": LBM_COLLISION_REG, "mrt": LBM_COLLISION_MRT}
LBM_KERNEL_TWO_LATTICE, LBM_KERNEL_AA_EVEN, LBM_KERNEL_AA_ODD, LBM_KERNEL_SNAPSHOT, LBM_KERNEL_MERGED, \
    LBM_KERNEL_KSTEP = 0, 1, 2, 3, 4, 5
KERNELS = {"two_lattice": LBM_KERNEL_TWO_LATTICE, "aa_even": LBM_KERNEL_AA_EVEN, "aa_odd": LBM_KERNEL_AA_ODD,
           "snapshot": LBM_KERNEL_SNAPSHOT, "merged": LBM_KERNEL_MERGED, "kstep": LBM_KERNEL_KSTEP}

STORAGE = {"f64": LBM_STORAGE_F64, "f32": LBM_STORAGE_F32, "f32s": LBM_STORAGE_F32S,
           "f16s": LBM_STORAGE_F16S, "bf16s": LBM_STORAGE_BF16S}
VARIANT = {"two_lattice": LBM_VARIANT_TWO_LATTICE, "aa": LBM_VARIANT_AA, "merged": LBM_VARIANT_MERGED,
           "kstep": LBM_VARIANT_KSTEP}
BC = {"periodic": LBM_BC_PERIODIC, "wall": LBM_BC_WALL, "lid": LBM_BC_LID}

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblbm_gb300.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "lbm.h")


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lbm_strerror(status)} (status {status})")


class lbm_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("face_bc", ctypes.c_int32 * 6),
        ("u_lid", ctypes.c_double * 3),
        ("rho_wall", ctypes.c_double),
        ("storage", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("force_mode", ctypes.c_int32),
        ("force_uniform", ctypes.c_double * 3),
        ("collision", ctypes.c_int32),
        ("trt_lambda", ctypes.c_double),
        ("mrt_s3", ctypes.c_double),
        ("mrt_s4", ctypes.c_double),
        ("lattice", ctypes.c_int32),
        ("sweep_steps", ctypes.c_int32),
    ]


_VP = ctypes.c_void_p
_H = ctypes.c_void_p
_CFGP = ctypes.POINTER(lbm_config)
_SIGNATURES = {
    "lbm_config_default": (None, [_CFGP]),
    "lbm_validate": (ctypes.c_int, [_CFGP]),
    "lbm_required_bytes": (ctypes.c_int, [_CFGP, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_create": (ctypes.c_int, [_CFGP, _VP, ctypes.POINTER(_H)]),
    "lbm_create_with_buffer": (ctypes.c_int, [_CFGP, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(_H)]),
    "lbm_destroy": (None, [_H]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_lattice": (ctypes.c_int, [_VP, _VP]),
    "lbm_lattice_q": (ctypes.c_int, [ctypes.c_int32, _VP, _VP]),
    "lbm_init_equilibrium": (ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32]),
    "lbm_set_force": (ctypes.c_int, [_H, _VP]),
    "lbm_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "lbm_time": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_moments": (ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32]),
    "lbm_populations": (ctypes.c_int, [_H, _VP, ctypes.c_int32]),
    "lbm_init_populations": (ctypes.c_int, [_H, _VP, ctypes.c_int32]),
    "lbm_reduce": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double)]),
    "lbm_reduce_populations": (ctypes.c_int, [_CFGP, _VP, ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_double),
                                              _VP]),
    "lbm_profile": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lbm_selftest_wait_timeout": (ctypes.c_int, [_H]),
    "lbm_profile_read": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double)]),
    "lbm_adjoint_step": (ctypes.c_int, [_H, _VP, _VP, _VP, ctypes.c_int32, _VP]),
    "lbm_adjoint_seed": (ctypes.c_int, [_H, _VP, _VP, _VP, ctypes.c_int32, _VP]),
    "lbm_adjoint_workspace_bytes": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_adjoint_forward": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_size_t]),
    "lbm_adjoint_backward": (ctypes.c_int, [_H, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_size_t]),
}

_lib = None
_lib_lock = threading.Lock()


def library() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2208_05429_gb300.build.build() "
                    "(there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def declared_symbols() -> list:
    """Names of the functions declared in include/lbm.h."""
    with open(HEADER_PATH) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _dtype_code(dtype) -> int:
    import torch
    if dtype == torch.float64:
        return LBM_DTYPE_F64
    if dtype == torch.float32:
        return LBM_DTYPE_F32
    raise ValueError(f"unsupported dtype {dtype}")


# ------------------------------------------------------------------ C names

def lbm_strerror(status: int) -> str:
    return library().lbm_strerror(int(status)).decode()


def lbm_config_default() -> lbm_config:
    c = lbm_config()
    library().lbm_config_default(ctypes.byref(c))
    return c


def lbm_validate(cfg: lbm_config) -> int:
    return library().lbm_validate(ctypes.byref(cfg))


def lbm_required_bytes(cfg: lbm_config) -> int:
    n = ctypes.c_size_t(0)
    _check(library().lbm_required_bytes(ctypes.byref(cfg), ctypes.byref(n)), "lbm_required_bytes")
    return n.value


def lbm_create(cfg: lbm_config, stream: int = 0):
    h = _H()
    _check(library().lbm_create(ctypes.byref(cfg), _VP(stream), ctypes.byref(h)), "lbm_create")
    return h


def lbm_create_with_buffer(cfg: lbm_config, stream: int, buffer_ptr: int, nbytes: int):
    h = _H()
    _check(library().lbm_create_with_buffer(ctypes.byref(cfg), _VP(stream), _VP(buffer_ptr), nbytes,
                                            ctypes.byref(h)), "lbm_create_with_buffer")
    return h


def lbm_destroy(h) -> None:
    library().lbm_destroy(h)


def lbm_lattice() -> Tuple[np.ndarray, np.ndarray]:
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    _check(library().lbm_lattice(c.ctypes.data, w.ctypes.data), "lbm_lattice")
    return c.astype(np.int64), w


def lbm_lattice_q(q: int) -> Tuple[np.ndarray, np.ndarray]:
    """c[q, 3], w[q] of lattice D3Q<q> (15, 19 or 27) in the library's order."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    _check(library().lbm_lattice_q(int(q), c.ctypes.data, w.ctypes.data), "lbm_lattice_q")
    return c.astype(np.int64), w


def lbm_init_equilibrium(h, rho=None, u=None, dtype_code: int = LBM_DTYPE_F32):
    _check(library().lbm_init_equilibrium(h, _ptr(rho), _ptr(u), dtype_code), "lbm_init_equilibrium")


def lbm_set_force(h, F):
    _check(library().lbm_set_force(h, _ptr(F)), "lbm_set_force")


def lbm_step(h, n: int):
    _check(library().lbm_step(h, int(n)), "lbm_step")


def lbm_time(h) -> int:
    t = ctypes.c_int64(0)
    _check(library().lbm_time(h, ctypes.byref(t)), "lbm_time")
    return t.value


def lbm_moments(h, rho, u, dtype_code: int):
    _check(library().lbm_moments(h, _ptr(rho), _ptr(u), dtype_code), "lbm_moments")


def lbm_populations(h, f_out, dtype_code: int):
    _check(library().lbm_populations(h, _ptr(f_out), dtype_code), "lbm_populations")


def lbm_init_populations(h, f_in, dtype_code: int):
    _check(library().lbm_init_populations(h, _ptr(f_in), dtype_code), "lbm_init_populations")


def lbm_reduce(h, raise_nonfinite: bool = True) -> np.ndarray:
    out = (ctypes.c_double * 5)()
    rc = library().lbm_reduce(h, out)
    if rc != LBM_OK and (raise_nonfinite or rc != LBM_ENONFINITE):
        raise LbmError(rc, "lbm_reduce")
    return np.array(out[:], dtype=np.float64)


def lbm_reduce_populations(cfg: lbm_config, f, F=None, stream: int = 0, raise_nonfinite: bool = True):
    """Sums of lbm_reduce() for canonical populations f (a CUDA tensor),
    without any device allocation (scratch in a fixed device array)."""
    out = (ctypes.c_double * 5)()
    rc = library().lbm_reduce_populations(ctypes.byref(cfg), _ptr(f), _dtype_code(f.dtype), _ptr(F), out,
                                          _VP(stream))
    if rc != LBM_OK and (raise_nonfinite or rc != LBM_ENONFINITE):
        raise LbmError(rc, "lbm_reduce_populations")
    return np.array(out[:], dtype=np.float64)


def lbm_profile(h, enable: bool):
    _check(library().lbm_profile(h, 1 if enable else 0), "lbm_profile")


def lbm_profile_read(h, kernel: int) -> Tuple[int, float]:
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(library().lbm_profile_read(h, int(kernel), ctypes.byref(n), ctypes.byref(ms)), "lbm_profile_read")
    return n.value, ms.value


def lbm_selftest_wait_timeout(h) -> int:
    """Status code of the wait-timeout self-test (LBM_ETIMEOUT expected)."""
    return int(library().lbm_selftest_wait_timeout(h))


def lbm_adjoint_step(h, f_t, lam_in, lam_out, dtype_code: int, dLdF=None):
    _check(library().lbm_adjoint_step(h, _ptr(f_t), _ptr(lam_in), _ptr(lam_out), dtype_code, _ptr(dLdF)),
           "lbm_adjoint_step")


def lbm_adjoint_seed(h, dLdrho, dLdu, lam, dtype_code: int, dLdF=None):
    _check(library().lbm_adjoint_seed(h, _ptr(dLdrho), _ptr(dLdu), _ptr(lam), dtype_code, _ptr(dLdF)),
           "lbm_adjoint_seed")


def lbm_adjoint_workspace_bytes(h, T: int, K: int) -> int:
    n = ctypes.c_size_t(0)
    _check(library().lbm_adjoint_workspace_bytes(h, int(T), int(K), ctypes.byref(n)),
           "lbm_adjoint_workspace_bytes")
    return n.value


def lbm_adjoint_forward(h, T: int, K: int, work, nbytes: int):
    _check(library().lbm_adjoint_forward(h, int(T), int(K), _ptr(work), nbytes), "lbm_adjoint_forward")


def lbm_adjoint_backward(h, dLdrho, dLdu, dtype_code: int, dLdf0, dLdF, work, nbytes: int):
    _check(library().lbm_adjoint_backward(h, _ptr(dLdrho), _ptr(dLdu), dtype_code, _ptr(dLdf0), _ptr(dLdF),
                                          _ptr(work), nbytes), "lbm_adjoint_backward")


# ------------------------------------------------------------------ wrapper

def make_config(shape: Sequence[int], tau: float, bc: Sequence[Union[str, int]] = ("periodic",) * 6,
                u_lid=(0.0, 0.0, 0.0), rho_wall: float = 1.0, storage: str = "f32", variant: str = "aa",
                force_mode: int = LBM_FORCE_NONE, force_uniform=(0.0, 0.0, 0.0),
                collision: Union[str, int] = "bgk", trt_lambda: float = 3.0 / 16.0,
                mrt_s3: float = 1.0, mrt_s4: float = 1.0, lattice: int = 19, sweep_steps: int = 0) -> lbm_config:
    """Build an lbm_config; shape is (nx, ny, nz), bc lists x-, x+, y-, y+, z-, z+;
    lattice is 15, 19 or 27 (D3Q15, D3Q19, D3Q27); sweep_steps the steps per
    sweep of the "kstep" variant (3 or 4; 0 = 3)."""
    c = lbm_config()
    c.nx, c.ny, c.nz = (int(v) for v in shape)
    c.tau = float(tau)
    for k in range(6):
        b = bc[k]
        c.face_bc[k] = BC[b] if isinstance(b, str) else int(b)
    for a in range(3):
        c.u_lid[a] = float(u_lid[a])
        c.force_uniform[a] = float(force_uniform[a])
    c.rho_wall = float(rho_wall)
    c.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    c.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
    c.force_mode = int(force_mode)
    c.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    c.trt_lambda = float(trt_lambda)
    c.mrt_s3, c.mrt_s4 = float(mrt_s3), float(mrt_s4)
    c.lattice = int(lattice)
    c.sweep_steps = int(sweep_steps)
    return c


CAVITY_BC = ("wall", "wall", "wall", "wall", "wall", "lid")


class Lattice:
    """One D3Q19 (or D3Q15 / D3Q27: ``lattice=15`` / ``27``) lattice on a GPU,
    memory owned by a torch tensor.

    force: None (no force), a 3-sequence (uniform force), or a float32 CUDA
    tensor [3, nz, ny, nx] (per-cell force field, kept alive here).
    """

    def __init__(self, shape, tau: float, bc=("periodic",) * 6, u_lid=(0.0, 0.0, 0.0), rho_wall: float = 1.0,
                 storage: str = "f32", variant: str = "aa", force=None, device=None, stream=None,
                 collision: str = "bgk", trt_lambda: float = 3.0 / 16.0, mrt_s3: float = 1.0,
                 mrt_s4: float = 1.0, lattice: int = 19, sweep_steps: int = 0):
        import torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if force is None:
            fm, fu = LBM_FORCE_NONE, (0.0, 0.0, 0.0)
        elif isinstance(force, torch.Tensor):
            fm, fu = LBM_FORCE_FIELD, (0.0, 0.0, 0.0)
        else:
            fm, fu = LBM_FORCE_UNIFORM, tuple(float(v) for v in force)
        self.cfg = make_config(shape, tau, bc, u_lid, rho_wall, storage, variant, fm, fu, collision, trt_lambda,
                               mrt_s3, mrt_s4, lattice, sweep_steps)
        self.q = int(lattice) or Q
        self.shape = tuple(int(v) for v in shape)  # (nx, ny, nz)
        self.nbytes = lbm_required_bytes(self.cfg)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._buf = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.h = lbm_create_with_buffer(self.cfg, self.stream.cuda_stream, self._buf.data_ptr(), self.nbytes)
        self._force = None
        self._work = None
        if fm == LBM_FORCE_FIELD:
            self.set_force(force)

    # canonical field shapes
    @property
    def field_shape(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def _empty(self, lead, dtype):
        import torch
        return torch.empty((*lead, *self.field_shape), dtype=dtype, device=self.device)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_force(self, F):
        import torch
        F = F.to(device=self.device, dtype=torch.float32).contiguous()
        assert tuple(F.shape) == (3, *self.field_shape)
        self._force = F
        lbm_set_force(self.h, F)

    def init_equilibrium(self, rho=None, u=None):
        import torch
        dt = torch.float64 if (rho is not None and rho.dtype == torch.float64) or \
            (u is not None and u.dtype == torch.float64) else torch.float32
        r = None if rho is None else rho.to(self.device, dt).contiguous()
        v = None if u is None else u.to(self.device, dt).contiguous()
        lbm_init_equilibrium(self.h, r, v, _dtype_code(dt))
        self._keep = (r, v)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    @property
    def time(self) -> int:
        return lbm_time(self.h)

    def moments(self, dtype=None):
        import torch
        dtype = dtype or torch.float32
        rho = self._empty((), dtype)
        u = self._empty((3,), dtype)
        lbm_moments(self.h, rho, u, _dtype_code(dtype))
        return rho, u

    def populations(self, dtype=None):
        import torch
        dtype = dtype or torch.float32
        f = self._empty((self.q,), dtype)
        lbm_populations(self.h, f, _dtype_code(dtype))
        return f

    def init_populations(self, f):
        if tuple(f.shape) != (self.q,) + self.field_shape:
            raise ValueError(f"populations of shape {tuple(f.shape)}: expected {(self.q,) + self.field_shape}")
        f = f.to(self.device).contiguous()
        lbm_init_populations(self.h, f, _dtype_code(f.dtype))
        self._keep = f

    def reduce(self, raise_nonfinite: bool = True) -> np.ndarray:
        return lbm_reduce(self.h, raise_nonfinite)

    def profile(self, enable: bool = True):
        """Start (clearing earlier records) or stop per-kernel event timing."""
        lbm_profile(self.h, enable)

    def profile_read(self) -> dict:
        """{kernel class: (launches, total device ms)} since profiling started."""
        out = {}
        for name, k in KERNELS.items():
            n, ms = lbm_profile_read(self.h, k)
            if n:
                out[name] = (n, ms)
        return out

    def selftest_wait_timeout(self) -> int:
        """MERGED with the neighbour-synchronised sweep only: run one sweep in
        which one tile never announces its progress, so that the bounded
        waits for it run out; return the recorded status (LBM_ETIMEOUT
        expected).  The populations are undefined afterwards."""
        return lbm_selftest_wait_timeout(self.h)

    # adjoint --------------------------------------------------------------
    def adjoint_step(self, f_t, lam_in, lam_out, dLdF=None):
        lbm_adjoint_step(self.h, f_t, lam_in, lam_out, _dtype_code(f_t.dtype), dLdF)

    def adjoint_seed(self, dLdu, dLdrho=None, dLdF=None, dtype=None):
        import torch
        dtype = dtype or dLdu.dtype
        lam = self._empty((Q,), dtype)
        lbm_adjoint_seed(self.h, None if dLdrho is None else dLdrho.to(dtype).contiguous(),
                         dLdu.to(dtype).contiguous(), lam, _dtype_code(dtype), dLdF)
        return lam

    def adjoint_forward(self, T: int, K: int):
        import torch
        nbytes = lbm_adjoint_workspace_bytes(self.h, T, K)
        self._work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        lbm_adjoint_forward(self.h, T, K, self._work, nbytes)

    def adjoint_backward(self, dLdu, dLdrho=None, dtype=None):
        """(dL/df^0 [19, ...], dL/dF [3, ...] float64) for the last adjoint_forward."""
        import torch
        dtype = dtype or dLdu.dtype
        dLdf0 = self._empty((Q,), dtype)
        dLdF = torch.zeros((3, *self.field_shape), dtype=torch.float64, device=self.device)
        lbm_adjoint_backward(self.h, None if dLdrho is None else dLdrho.to(dtype).contiguous(),
                             dLdu.to(dtype).contiguous(), _dtype_code(dtype), dLdf0, dLdF,
                             self._work, self._work.numel())
        return dLdf0, dLdF
