"""Reduced-precision storage: the velocity error against an FP64 run of the
same case is measured and held under the bound stated here.  Workload: the
periodic Taylor-Green box of the precision study (U0 = 0.04, tau = 0.52), at
64^3 for 400 steps (the 512^3 x 2000-step case is run by bench.py's precision
mode); FP32 arithmetic in every format.

Bounds (relative max-norm of u vs FP64), about twice the measured errors
(F32 1.27e-5, F32S 1.24e-5, F16S 1.07e-3, BF16S 5.6e-3): F32 2.5e-5, F32S
2.5e-5, F16S 2.2e-3, BF16S 1.2e-2.  FP16/BF16 parity is not pinned to the
oracle beyond this measured bound."""
import numpy as np
import pytest

from paper_2208_05429_gb300 import inputs
from paper_2208_05429_gb300.lbm import Lattice

pytestmark = pytest.mark.gpu

BOUNDS = {"f32": 2.5e-5, "f32s": 2.5e-5, "f16s": 2.2e-3, "bf16s": 1.2e-2}


def _tg(storage, n=64, steps=400, variant="merged"):
    import torch
    lat = Lattice((n, n, n), 0.52, storage=storage, variant=variant)
    u0 = torch.tensor(inputs.taylor_green_velocity(n, n, n, 0.04))
    lat.init_equilibrium(None, u0.to(lat.device))
    lat.step(steps)
    _, u = lat.moments(torch.float64)
    ke = lat.reduce()[4]
    return u.cpu().numpy(), ke


def test_reduced_precision_error_bounds(gpu):
    u64, ke64 = _tg("f64")
    errs = {}
    for s, bound in BOUNDS.items():
        u, ke = _tg(s)
        err = float(np.max(np.abs(u - u64)) / np.max(np.abs(u64)))
        errs[s] = err
        print(f"storage {s}: max-norm u error vs FP64 {err:.3e}; KE rel err {abs(ke - ke64) / ke64:.3e}")
    for s, bound in BOUNDS.items():
        assert errs[s] <= bound, (s, errs[s])
    # shifted storage must not be worse than plain FP32
    assert errs["f32s"] <= errs["f32"] * 1.5
