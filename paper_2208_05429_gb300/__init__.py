"""GB300-native D3Q19 lattice Boltzmann hot path (Fu & Song, arXiv 2208.05429).

The compute runs in the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); this package holds its ctypes binding (:mod:`.lbm`), the
autograd bridge of the adjoint (:mod:`.autograd`), the seeded input
generators (:mod:`.inputs`) and the build script (:mod:`.build`).
"""
from .lbm import (  # noqa: F401
    CAVITY_BC, LBM_BC_LID, LBM_BC_PERIODIC, LBM_BC_WALL, Lattice, LbmError, library, lbm_lattice,
    make_config,
)
