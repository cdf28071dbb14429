"""16-bit storage (F16S, BF16S) against the FP64 oracle with the same
storage rounding, element by element.

The GPU keeps each population as s_i = f_i - w_i in binary16 or bfloat16,
rounded to nearest-even once per time step, with the collision in FP32 in
between.  The expected state is the oracle's FP64 step followed by
oracle.store_round after every step, decoded the way the GPU decodes it
(w_i + s_i in FP32).  Two effects separate them: where the FP32 and FP64
collisions straddle a rounding boundary the stored values are one storage
ulp apart, and where s_i is so small that the storage ulp is below the FP32
collision's own rounding error (a few 1e-8 absolute) they differ by that
error.  So one step, taken from the GPU's own state, keeps every value
within one storage ulp plus 4e-8 of the expected one and leaves at least 99%
of them equal.  A merged sweep does two steps without exposing the first:
a one-ulp difference after the first step then reaches the second step's
outputs through the collision, up to one storage ulp of the largest value,
so the bound for the sweep is two ulps plus that plus 1e-7 (98% equal)."""
import numpy as np
import pytest

import oracle
from gpu_cases import cases, gpu_state, load_state, make_gpu, oracle_force_as_f32, start_state

pytestmark = pytest.mark.gpu

NAMES = ["channel_37x19x23", "periodic_field_20x18x17", "mixed_33x40x9", "narrow_2x21x5", "cavity16"]


def _ulp(s, storage):
    a = np.abs(s)
    if storage == "f16s":
        u = np.spacing(a.astype(np.float16)).astype(np.float64)
    else:
        _, e = np.frexp(a)
        u = np.ldexp(1.0, e - 8)
    return np.maximum(u, 2.0 ** -133)


def _decoded(s_exp, w32):
    """The populations the GPU reports for stored shifted values s (its FP32
    decode, w_i + s_i)."""
    return (s_exp.astype(np.float32) + w32).astype(np.float64)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("name", NAMES)
def test_aa_steps_within_one_storage_ulp(gpu, storage, name):
    """Two AA steps (even, then odd), each against the oracle stepping the
    GPU's own state once."""
    _, w, _ = oracle.lattice()
    w32 = w.astype(np.float32)[:, None, None, None]
    cfg = oracle_force_as_f32(cases()[name])
    f0, _ = oracle.store_round(start_state(cfg, seed=21), storage)
    lat = make_gpu(cfg, storage, "aa")
    load_state(lat, f0)
    prev = f0
    for step in (1, 2):
        lat.step(1)
        _, s_exp = oracle.store_round(oracle.run(cfg, prev, 1), storage)
        got = gpu_state(lat)
        diff = np.abs(got - _decoded(s_exp, w32))
        bound = _ulp(s_exp, storage) + 4e-8
        frac = float(np.mean(diff == 0.0))
        print(f"{name} {storage} aa step {step}: max {np.max(diff / bound):.3f} of the bound, {100 * frac:.2f}% equal")
        assert np.all(diff <= bound) and frac >= 0.99
        prev = got


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("name", NAMES)
def test_merged_sweep_within_storage_ulps(gpu, storage, name):
    _, w, _ = oracle.lattice()
    w32 = w.astype(np.float32)[:, None, None, None]
    cfg = oracle_force_as_f32(cases()[name])
    f0, _ = oracle.store_round(start_state(cfg, seed=22), storage)
    lat = make_gpu(cfg, storage, "merged")
    load_state(lat, f0)
    lat.step(2)
    f1, _ = oracle.store_round(oracle.run(cfg, f0, 1), storage)
    _, s_exp = oracle.store_round(oracle.run(cfg, f1, 1), storage)
    diff = np.abs(gpu_state(lat) - _decoded(s_exp, w32))
    bound = 2.0 * _ulp(s_exp, storage) + _ulp(np.max(np.abs(s_exp)), storage) + 1e-7
    frac = float(np.mean(diff == 0.0))
    print(f"{name} {storage} merged sweep: max {np.max(diff / bound):.3f} of the bound, {100 * frac:.2f}% equal")
    assert np.all(diff <= bound) and frac >= 0.98
