"""torch.autograd bridge of the hand-written adjoint kernels.

``LBMFunction.apply(f0, F, lattice, T, K)`` runs T time steps of ``lattice``
(a :class:`~paper_2208_05429_gb300.lbm.Lattice` created with a per-cell force
field) from the populations f0 under the body force F, and returns the
velocity field u^T [3, nz, ny, nx].  Its backward pass seeds the adjoint with
dL/du^T, recomputes each K-step segment from a checkpoint and runs the
reverse collide-stream kernel, returning dL/df0 and dL/dF (accumulated in
FP64 on the device, returned in F's dtype).  All the work is done by the C
ABI calls lbm_adjoint_forward / lbm_adjoint_backward.
"""
from __future__ import annotations

import torch

from .lbm import Lattice


class LBMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0: torch.Tensor, F: torch.Tensor, lattice: Lattice, T: int, K: int):
        lattice.set_force(F.detach())
        lattice.init_populations(f0.detach())
        lattice.adjoint_forward(int(T), int(K))
        _, u = lattice.moments(f0.dtype)
        ctx.lattice = lattice
        ctx.f_dtype = f0.dtype
        ctx.F_dtype = F.dtype
        return u

    @staticmethod
    def backward(ctx, grad_u: torch.Tensor):
        dLdf0, dLdF = ctx.lattice.adjoint_backward(grad_u.contiguous(), dtype=ctx.f_dtype)
        return dLdf0, dLdF.to(ctx.F_dtype), None, None, None


def simulate(f0: torch.Tensor, F: torch.Tensor, lattice: Lattice, T: int, K: int = 20) -> torch.Tensor:
    """u^T as a differentiable function of (f0, F)."""
    return LBMFunction.apply(f0, F, lattice, T, K)
