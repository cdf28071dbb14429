"""lbm_reduce_populations(): the reduction for callers that cannot allocate
device memory (a caching allocator holding the free memory, a loop that must
not take cudaMalloc's device synchronisation, an allocator callback).

It keeps its scratch in a fixed device array instead of a handle's buffer.
Checked here through the C ABI: on two calls in a row (the second sees the
scratch the first left behind) its sums equal lbm_reduce() on the handle
that produced the populations, within the tolerances of the FP64 reduction
tests (mass 1e-13 relative, momentum 1e-11 of its largest component, kinetic
energy 1e-11 relative).  The file name sorts last, so a run that stops at
the first failure has run every other test before this one.
"""
import numpy as np
import pytest

import oracle
from gpu_cases import cases, load_state, make_gpu, oracle_force_as_f32, start_state

pytestmark = pytest.mark.gpu


def _close(got, exp):
    assert abs(got[0] - exp[0]) <= 1e-13 * abs(exp[0])
    scale = max(np.max(np.abs(exp[1:4])), 1e-300)
    assert np.max(np.abs(got[1:4] - exp[1:4])) <= 1e-11 * scale + 1e-15
    assert abs(got[4] - exp[4]) <= 1e-11 * abs(exp[4]) + 1e-18


@pytest.mark.parametrize("name,storage", [("channel_37x19x23", "f64"), ("periodic_field_20x18x17", "f64"),
                                          ("cavity16", "f32"), ("mixed_33x40x9", "f32")])
def test_reduce_without_allocation_matches_lbm_reduce(gpu, name, storage):
    import torch
    from paper_2208_05429_gb300 import lbm
    cfg = oracle_force_as_f32(cases()[name])
    lat = make_gpu(cfg, storage, "aa")
    load_state(lat, start_state(cfg, seed=3))
    dt = torch.float64 if storage == "f64" else torch.float32
    F = lat._force
    stream = lat.stream.cuda_stream
    for nsteps in (3, 4):  # the second call starts from the first one's scratch
        lat.step(nsteps)
        exp = lat.reduce()
        f = lat.populations(dt)
        got = lbm.lbm_reduce_populations(lat.cfg, f, F=F, stream=stream)
        _close(got, exp)
    lat.close()


def test_reduce_without_allocation_flags_nonfinite_then_clears(gpu):
    import torch
    from paper_2208_05429_gb300 import lbm
    cfg = oracle.cavity(12, 0.6)
    lat = make_gpu(cfg, "f32", "aa")
    load_state(lat, start_state(cfg))
    exp = lat.reduce()
    f = lat.populations(torch.float32)
    bad = f.clone()
    bad[3, 4, 5, 6] = float("nan")
    stream = lat.stream.cuda_stream
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_reduce_populations(lat.cfg, bad, stream=stream)
    assert ei.value.status == lbm.LBM_ENONFINITE
    # the next call clears the flag the previous one left set
    _close(lbm.lbm_reduce_populations(lat.cfg, f, stream=stream), exp)
    lat.close()
