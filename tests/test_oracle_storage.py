"""Pins of oracle.store_round, the 16-bit shifted storage the GPU's F16S and
BF16S formats hold (s_i = f_i - w_i rounded to nearest-even): against torch's
own float16 / bfloat16 conversions (round-to-nearest-even), exact ties, and
idempotence."""
import numpy as np
import pytest

import oracle


def _f(seed):
    rng = np.random.default_rng(seed)
    cfg = oracle.Config(nx=5, ny=4, nz=3, tau=0.7)
    return oracle.init_equilibrium(cfg) * (1.0 + 0.05 * rng.standard_normal((19, 3, 4, 5)))


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_store_round_matches_torch(storage):
    import torch
    _, w, _ = oracle.lattice()
    f = _f(1)
    got_f, got_s = oracle.store_round(f, storage)
    s = f - w[:, None, None, None]
    t = torch.tensor(s.astype(np.float32) if storage == "bf16s" else s)
    ref = t.to(torch.float16 if storage == "f16s" else torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got_s, ref)
    assert np.allclose(got_f - w[:, None, None, None], got_s, rtol=0, atol=1e-18)
    again_f, again_s = oracle.store_round(got_f, storage)
    assert np.array_equal(again_s, got_s)


def test_store_round_ties_to_even():
    _, w, _ = oracle.lattice()
    one = np.zeros((19, 1)) + w[:, None]
    # bfloat16: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> 1 (even); 1 + 3 * 2^-8 -> 1 + 2^-6
    _, s = oracle.store_round(one + (1.0 + 2.0 ** -8), "bf16s")
    assert np.all(s == 1.0)
    _, s = oracle.store_round(one + (1.0 + 3 * 2.0 ** -8), "bf16s")
    assert np.all(s == 1.0 + 2.0 ** -6)
    # binary16: 1 + 2^-11 is a tie -> 1; 1 + 3 * 2^-11 -> 1 + 2^-9
    _, s = oracle.store_round(one + (1.0 + 2.0 ** -11), "f16s")
    assert np.all(s == 1.0)
    _, s = oracle.store_round(one + (1.0 + 3 * 2.0 ** -11), "f16s")
    assert np.all(s == 1.0 + 2.0 ** -9)
