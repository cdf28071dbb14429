"""The C-ABI library loads, exports every symbol include/lbm.h declares and
validates configurations on the host (no GPU needed)."""
import ctypes

import numpy as np
import pytest

from paper_2208_05429_gb300 import lbm


def test_every_declared_symbol_is_exported(cuda_lib):
    names = lbm.declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(cuda_lib, n)]
    assert not missing, missing
    # and the binding wraps each of them
    assert set(names) <= set(lbm._SIGNATURES)


def test_lattice_table(cuda_lib):
    c, w = lbm.lbm_lattice()
    vecs = {tuple(v) for v in c}
    assert len(vecs) == 19 and tuple(c[0]) == (0, 0, 0)
    assert all(max(abs(v) for v in cv) <= 1 and sum(a * a for a in cv) <= 2 for cv in vecs)
    for i in range(1, 10):
        assert next(v for v in c[i] if v != 0) == -1
        assert np.array_equal(c[i + 9], -c[i])
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3, atol=1e-16)


@pytest.mark.parametrize("q", [15, 27])
def test_other_lattice_tables(cuda_lib, q):
    """D3Q15 / D3Q27: the admitted vectors, the half-neighbour order, and the
    weights from the moment identities (up to fourth order; for D3Q27 the
    D1Q3 product rule sum w cx^2 cy^2 cz^2 = 1/27)."""
    import itertools
    c, w = lbm.lbm_lattice_q(q)
    norms = {15: {0, 1, 3}, 27: {0, 1, 2, 3}}[q]
    vecs = [tuple(int(a) for a in v) for v in c]
    assert set(vecs) == {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) in norms}
    h = (q - 1) // 2
    assert vecs[0] == (0, 0, 0)
    for i in range(1, h + 1):
        assert next(a for a in vecs[i] if a != 0) == -1
        assert np.array_equal(c[i + h], -c[i])
    assert vecs[1:h + 1] == sorted(vecs[1:h + 1])       # lexicographic within the half
    cf = c.astype(np.float64)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("q,qa,qb->ab", w, cf, cf), np.eye(3) / 3, atol=1e-16)
    assert abs(np.sum(w * cf[:, 0] ** 2 * cf[:, 1] ** 2) - 1.0 / 9.0) < 1e-16
    if q == 27:
        assert abs(np.sum(w * cf[:, 0] ** 2 * cf[:, 1] ** 2 * cf[:, 2] ** 2) - 1.0 / 27.0) < 1e-16
    with pytest.raises(lbm.LbmError):
        lbm.lbm_lattice_q(21)
    # the 19-velocity query is lbm_lattice's table
    assert np.array_equal(lbm.lbm_lattice_q(19)[0], lbm.lbm_lattice()[0])


@pytest.mark.parametrize("q", [15, 27])
def test_other_lattices_validate(cuda_lib, q):
    for variant in ("aa", "two_lattice", "merged"):
        for storage in ("f64", "f32", "f32s", "f16s", "bf16s"):
            for coll in ("bgk", "trt", "reg"):
                cfg = lbm.make_config((16, 16, 16), 0.7, lbm.CAVITY_BC, storage=storage, variant=variant,
                                      collision=coll, lattice=q)
                assert lbm.lbm_validate(cfg) == lbm.LBM_OK, (variant, storage, coll)
    cfg = lbm.make_config((16, 16, 16), 0.7, collision="mrt", lattice=q)
    assert lbm.lbm_validate(cfg) == lbm.LBM_EUNSUPPORTED
    pop = q * 64 ** 3 * 4
    aa = lbm.make_config((64, 64, 64), 0.6, storage="f32", variant="aa", lattice=q)
    mg = lbm.make_config((64, 64, 64), 0.6, lbm.CAVITY_BC, storage="f32", variant="merged", lattice=q)
    assert pop <= lbm.lbm_required_bytes(aa) < pop * 1.01
    assert pop <= lbm.lbm_required_bytes(mg) < pop * 1.01      # MERGED runs the AA pair: no shadow
    for bad in (21, 9, -1):
        cfg = lbm.make_config((16, 16, 16), 0.7, lattice=bad)
        assert lbm.lbm_validate(cfg) == lbm.LBM_EINVAL


def test_kstep_validation(cuda_lib):
    """The K-step sweep: 3 or 4 steps, FP32-compute storage, D3Q19, BGK;
    two lattices of memory."""
    for st in ("f32", "f32s", "f16s", "bf16s"):
        for k in (0, 3, 4):
            cfg = lbm.make_config((24, 20, 12), 0.7, lbm.CAVITY_BC, storage=st, variant="kstep", sweep_steps=k)
            assert lbm.lbm_validate(cfg) == lbm.LBM_OK, (st, k)
    for kw in (dict(storage="f64"), dict(lattice=27), dict(collision="trt"), dict(collision="mrt")):
        cfg = lbm.make_config((16, 16, 16), 0.7, variant="kstep", **kw)
        assert lbm.lbm_validate(cfg) == lbm.LBM_EUNSUPPORTED, kw
    pop = 19 * 64 ** 3 * 4
    ks = lbm.make_config((64, 64, 64), 0.6, storage="f32", variant="kstep")
    assert 2 * pop <= lbm.lbm_required_bytes(ks) < 2 * pop * 1.01
    assert lbm.lbm_config_default().sweep_steps == 0


def test_lattice_table_is_the_one_the_schedule_tests_restate(cuda_lib):
    from test_merged_schedule import GPU_C
    c, _ = lbm.lbm_lattice()
    assert [tuple(int(v) for v in row) for row in c] == GPU_C


def test_default_config_valid(cuda_lib):
    cfg = lbm.lbm_config_default()
    assert (cfg.nx, cfg.ny, cfg.nz) == (32, 32, 32)
    assert lbm.lbm_validate(cfg) == lbm.LBM_OK
    assert lbm.lbm_required_bytes(cfg) >= 19 * 32 ** 3 * 4


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("ny", -3), ("nz", 70000), ("tau", 0.5), ("tau", float("nan")), ("rho_wall", 0.0),
    ("storage", 9), ("variant", 4), ("variant", 5), ("variant", -1), ("force_mode", 5), ("sweep_steps", 2),
    ("sweep_steps", 5),
    ("collision", 4), ("collision", -1), ("mrt_s3", 0.0), ("mrt_s4", 2.0), ("trt_lambda", 0.0), ("trt_lambda", float("inf")),
])
def test_invalid_configs_rejected(cuda_lib, field, value):
    cfg = lbm.lbm_config_default()
    setattr(cfg, field, value)
    assert lbm.lbm_validate(cfg) == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm_required_bytes(cfg)


def test_invalid_faces_and_lid(cuda_lib):
    cfg = lbm.lbm_config_default()
    cfg.face_bc[0] = lbm.LBM_BC_WALL  # x- wall with x+ periodic
    assert lbm.lbm_validate(cfg) == lbm.LBM_EINVAL
    cfg = lbm.make_config((8, 8, 8), 0.6, lbm.CAVITY_BC, u_lid=(0.3, 0.0, 0.0))
    assert lbm.lbm_validate(cfg) == lbm.LBM_EINVAL
    cfg = lbm.make_config((2000, 2000, 2000), 0.6)
    assert lbm.lbm_validate(cfg) == lbm.LBM_EINVAL


def test_required_bytes_scale(cuda_lib):
    aa = lbm.make_config((64, 64, 64), 0.6, storage="f32", variant="aa")
    tl = lbm.make_config((64, 64, 64), 0.6, storage="f32", variant="two_lattice")
    mg = lbm.make_config((64, 64, 64), 0.6, storage="f32", variant="merged")
    h16 = lbm.make_config((64, 64, 64), 0.6, storage="f16s", variant="aa")
    pop = 19 * 64 ** 3 * 4
    assert pop <= lbm.lbm_required_bytes(aa) < pop * 1.01
    assert 2 * pop <= lbm.lbm_required_bytes(tl) < 2 * pop * 1.01
    assert pop < lbm.lbm_required_bytes(mg) < 1.6 * pop
    assert pop // 2 <= lbm.lbm_required_bytes(h16) < pop


def test_every_collision_on_every_schedule(cuda_lib):
    for variant in ("aa", "two_lattice", "merged"):
        for coll in ("bgk", "trt", "reg", "mrt"):
            cfg = lbm.make_config((16, 16, 16), 0.7, lbm.CAVITY_BC, storage="f32", variant=variant, collision=coll)
            assert lbm.lbm_validate(cfg) == lbm.LBM_OK, (variant, coll)
    assert lbm.lbm_config_default().collision == lbm.LBM_COLLISION_BGK


def test_strerror(cuda_lib):
    assert lbm.lbm_strerror(0) == "success"
    assert "non-finite" in lbm.lbm_strerror(lbm.LBM_ENONFINITE)
    assert lbm.lbm_strerror(12345) == "unknown status"


def test_config_struct_layout_matches_header(cuda_lib):
    """The ctypes mirror of lbm_config has the C layout (checked through a
    round trip: lbm_config_default writes every field)."""
    assert ctypes.sizeof(lbm.lbm_config) == 168
    cfg = lbm.lbm_config_default()
    assert cfg.tau == 0.6 and cfg.rho_wall == 1.0 and list(cfg.face_bc) == [0] * 6
    assert cfg.storage == lbm.LBM_STORAGE_F32 and cfg.variant == lbm.LBM_VARIANT_AA
    assert cfg.collision == lbm.LBM_COLLISION_BGK and cfg.trt_lambda == 3.0 / 16.0
    assert cfg.lattice == lbm.LBM_LATTICE_D3Q19


def test_create_without_gpu_fails_cleanly(cuda_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = lbm.lbm_config_default()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(cfg, 0)


def test_required_bytes_merged_z_chunks(cuda_lib):
    """A 64^3 cavity gives the shadow-shell sweep 10 column tiles (32 x 14),
    fewer than the 152 SMs of a GB300 (the count assumed without a GPU), so
    z is split into chunks and the handle also holds the copy of the two
    planes next to every chunk boundary: 19 x 2 (nzc - 1) planes."""
    n, es, nsp, sms = 64, 4, 88, 152
    tiles = ((n + 31) // 32) * ((n + 13) // 14)

    def cost(k):
        return ((tiles * k + sms - 1) // sms) * (n / k + (3 if k > 1 else 0))

    nzc = min(range(1, n // 4 + 1), key=lambda k: (cost(k), k))
    if cost(nzc) > 0.95 * cost(1):
        nzc = 1
    assert nzc > 1
    pop = 19 * n ** 3 * es
    shadow = 2 * tiles * 19 * nsp * n * es
    zcopy = 19 * 2 * (nzc - 1) * n * n * es
    mg = lbm.make_config((n, n, n), 0.6, lbm.CAVITY_BC, u_lid=(0.05, 0.0, 0.0), storage="f32", variant="merged")
    extra = lbm.lbm_required_bytes(mg) - pop - shadow - zcopy
    assert 0 <= extra < 64 * 1024
