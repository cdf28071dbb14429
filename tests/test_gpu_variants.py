"""The schedules agree bit for bit (the paper verifies its two-step solvers
against the single-step ones, Sec. 5.1; here the check is exact):
TWO_LATTICE == AA == MERGED for every storage format, both two-step sweeps
of MERGED (neighbour-synchronised and shadow-shell, chosen with
LBM_MERGED_SWEEP when the handle is created), odd and even step counts and
mixed step(n) sequences."""
import numpy as np
import pytest

from gpu_cases import cases, load_state, make_gpu, oracle_force_as_f32, start_state

pytestmark = pytest.mark.gpu

CASES = cases()
STORAGES = ["f64", "f32", "f32s", "f16s", "bf16s"]


def _raw(lat):
    import torch
    return lat.populations(torch.float64)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nsteps", [5, 6])
def test_schedules_bitwise_equal(gpu, monkeypatch, storage, name, nsteps):
    """(Where a lattice has a periodic face, or the storage is FP64, the
    neighbour-synchronised sweep cannot run and the handle takes the
    shadow-shell one.)"""
    import torch
    cfg = oracle_force_as_f32(CASES[name])
    f0 = start_state(cfg, seed=3)
    ref = None
    runs = [("two_lattice", None), ("aa", None), ("merged", None), ("merged", "neighbour"), ("merged", "shadow")]
    for variant, sweep in runs:
        if sweep:
            monkeypatch.setenv("LBM_MERGED_SWEEP", sweep)
        lat = make_gpu(cfg, storage, variant)
        monkeypatch.delenv("LBM_MERGED_SWEEP", raising=False)
        load_state(lat, f0)
        lat.step(nsteps)
        got = _raw(lat)
        if ref is None:
            ref = got
        else:
            assert torch.equal(got, ref), (variant, sweep)
        rho, u = lat.moments(torch.float64)
        assert torch.isfinite(u).all()


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_mixed_step_sequences(gpu, storage):
    """MERGED stepped 1, 2, 3, 1, 2 steps at a time (crossing AA parities)
    equals AA stepped 9 times and TWO_LATTICE stepped one by one."""
    import torch
    cfg = oracle_force_as_f32(CASES["channel_37x19x23"])
    f0 = start_state(cfg, seed=9)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f0)
    a.step(9)
    m = make_gpu(cfg, storage, "merged")
    load_state(m, f0)
    for k in (1, 2, 3, 1, 2):
        m.step(k)
    t = make_gpu(cfg, storage, "two_lattice")
    load_state(t, f0)
    for _ in range(9):
        t.step(1)
    # shadow-shell sweep: consecutive sweeps reuse the shadow, a single step
    # in between invalidates it
    s3 = make_gpu(cfg, storage, "merged")
    load_state(s3, f0)
    for k in (2, 2, 1, 3, 1):
        s3.step(k)
    assert m.time == a.time == t.time == s3.time == 9
    ra, rm, rt, r3 = _raw(a), _raw(m), _raw(t), _raw(s3)
    assert torch.equal(ra, rm) and torch.equal(ra, rt) and torch.equal(ra, r3)
    # moments agree at both parities (a is at the odd parity after 9 steps)
    for lat in (a, m, t, s3):
        rho, u = lat.moments(torch.float64)
        r0, u0 = a.moments(torch.float64)
        assert torch.equal(rho, r0) and torch.equal(u, u0)


@pytest.mark.parametrize("storage", ["f32", "bf16s"])
def test_shadow_refreshed_after_new_state(gpu, storage):
    """A state installed between shadow-shell sweeps replaces the shadow:
    sweeps, a new state, sweeps again == AA on the new state."""
    import torch
    cfg = oracle_force_as_f32(CASES["mixed_33x40x9"])
    m = make_gpu(cfg, storage, "merged")
    load_state(m, start_state(cfg, seed=4))
    m.step(4)
    f1 = start_state(cfg, seed=5)
    load_state(m, f1)
    m.step(4)
    a = make_gpu(cfg, storage, "aa")
    load_state(a, f1)
    a.step(4)
    assert torch.equal(_raw(m), _raw(a))


def test_equilibrium_init_matches_oracle(gpu):
    import torch
    import oracle
    from paper_2208_05429_gb300 import inputs
    from gpu_cases import gpu_state
    from helpers import relmax
    cfg = oracle.Config(nx=24, ny=20, nz=18, tau=0.6)
    u0 = inputs.taylor_green_velocity(24, 20, 18, 0.04)
    rho0, _ = inputs.random_density_velocity(24, 20, 18, seed=2)
    ref = oracle.init_equilibrium(cfg, rho0, u0)
    lat = make_gpu(cfg, "f64", "aa")
    lat.init_equilibrium(torch.tensor(rho0, device=lat.device), torch.tensor(u0, device=lat.device))
    assert relmax(gpu_state(lat), ref) <= 1e-15


@pytest.mark.parametrize("variant", ["aa", "two_lattice", "merged"])
@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_graph_replay_matches_direct_launches(gpu, variant, storage):
    """step(n) with n >= 32 replays a captured CUDA graph of 32 time steps;
    it must equal stepping one time step per call (direct launches), also
    after the force field moves to new memory (the graph is rebuilt) and
    when the call starts at the odd AA parity."""
    import torch
    cfg = oracle_force_as_f32(CASES["channel_37x19x23"])
    f0 = start_state(cfg, seed=12)
    a = make_gpu(cfg, storage, variant)
    load_state(a, f0)
    a.step(1)           # odd parity for AA-based schedules
    a.step(70)          # two graph replays + direct tail
    a.step(64)          # cached graph reused
    b = make_gpu(cfg, storage, variant)
    load_state(b, f0)
    for _ in range(135):
        b.step(1)
    assert a.time == b.time == 135
    assert torch.equal(_raw(a), _raw(b))


def test_graph_rebuilt_after_force_field_change(gpu):
    import torch
    cfg = oracle_force_as_f32(CASES["periodic_field_20x18x17"])
    f0 = start_state(cfg, seed=13)
    F1 = torch.tensor(np.asarray(cfg.force_field, dtype=np.float32), device="cuda")
    F2 = (2.0 * F1).contiguous()
    a = make_gpu(cfg, "f32", "aa")
    a.set_force(F1)
    load_state(a, f0)
    a.step(32)
    a.set_force(F2)
    a.step(32)
    b = make_gpu(cfg, "f32", "aa")
    b.set_force(F1)
    load_state(b, f0)
    for _ in range(32):
        b.step(1)
    b.set_force(F2)
    for _ in range(32):
        b.step(1)
    assert torch.equal(_raw(a), _raw(b))


def test_bounded_wait_gives_up_and_reports(gpu, monkeypatch):
    """Failure detection of the inter-CTA waits of the neighbour-synchronised
    sweep: in a sweep where one tile never announces its progress, the
    tiles waiting for it give up after their bounded polls, so do the tiles
    waiting for those, and the sweep reports LBM_ETIMEOUT (no fault, no
    unbounded spin).  The handle keeps working afterwards: a new state steps
    exactly like AA.  Other handles and the odd parity are refused."""
    import torch
    from paper_2208_05429_gb300.lbm import LBM_ESTATE, LBM_ETIMEOUT
    cfg = oracle_force_as_f32(CASES["cavity16"])
    f0 = start_state(cfg, seed=21)
    monkeypatch.setenv("LBM_MERGED_SWEEP", "neighbour")
    w = make_gpu(cfg, "f32", "merged")
    monkeypatch.delenv("LBM_MERGED_SWEEP")
    load_state(w, f0)
    w.step(2)
    assert w.selftest_wait_timeout() == LBM_ETIMEOUT
    assert w.time == 2
    load_state(w, f0)
    w.step(4)
    a = make_gpu(cfg, "f32", "aa")
    load_state(a, f0)
    a.step(4)
    assert torch.equal(_raw(w), _raw(a))
    assert np.all(np.isfinite(w.reduce()))
    w.step(1)
    assert w.selftest_wait_timeout() == LBM_ESTATE   # odd parity
    assert a.selftest_wait_timeout() == LBM_ESTATE   # not a MERGED handle
    monkeypatch.setenv("LBM_MERGED_SWEEP", "shadow")
    s = make_gpu(cfg, "f32", "merged")
    monkeypatch.delenv("LBM_MERGED_SWEEP")
    assert s.selftest_wait_timeout() == LBM_ESTATE   # the shadow-shell sweep


def _random_config(rng):
    """A random small lattice: ragged against the 32-wide tiles and the
    14-row bands, random face types (periodic pairs, walls, lids) and force."""
    import oracle
    from oracle import BC_LID, BC_PERIODIC, BC_WALL, FORCE_NONE, FORCE_UNIFORM
    nx, ny, nz = (int(v) for v in rng.integers([1, 1, 2], [80, 48, 24]))
    bc = []
    for a in range(3):
        if rng.random() < 0.4:
            bc += [BC_PERIODIC, BC_PERIODIC]
        else:
            bc += [BC_LID if rng.random() < 0.3 else BC_WALL, BC_LID if rng.random() < 0.3 else BC_WALL]
    lid = tuple(float(v) for v in rng.uniform(-0.04, 0.04, 3))
    fm = FORCE_UNIFORM if rng.random() < 0.5 else FORCE_NONE
    fu = tuple(float(v) for v in rng.uniform(-2e-5, 2e-5, 3)) if fm == FORCE_UNIFORM else (0.0, 0.0, 0.0)
    return oracle.Config(nx=nx, ny=ny, nz=nz, tau=float(rng.uniform(0.52, 1.2)), bc=tuple(bc), u_lid=lid,
                         force_mode=fm, force_uniform=fu)


@pytest.mark.parametrize("seed", range(12))
def test_random_shapes_merged_equal_aa(gpu, monkeypatch, seed):
    import torch
    rng = np.random.default_rng(1000 + seed)
    cfg = _random_config(rng)
    storage = ["f64", "f32", "f32s", "f16s", "bf16s"][seed % 5]
    nsteps = int(rng.integers(2, 9))
    f0 = start_state(cfg, seed=seed)
    ref = make_gpu(cfg, storage, "aa")
    load_state(ref, f0)
    ref.step(nsteps)
    want = _raw(ref)
    for sweep in ("shadow", "neighbour"):
        monkeypatch.setenv("LBM_MERGED_SWEEP", sweep)
        lat = make_gpu(cfg, storage, "merged")
        monkeypatch.delenv("LBM_MERGED_SWEEP")
        load_state(lat, f0)
        lat.step(nsteps)
        assert torch.equal(_raw(lat), want), (sweep, cfg.nx, cfg.ny, cfg.nz, cfg.bc, storage, nsteps)


def _zchunk_config(shape):
    import oracle
    from oracle import BC_LID, BC_PERIODIC, BC_WALL, FORCE_UNIFORM
    nx, ny, nz = shape
    return oracle.Config(nx=nx, ny=ny, nz=nz, tau=0.7, bc=(BC_WALL, BC_WALL, BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_LID),
                         u_lid=(0.03, -0.01, 0.0), force_mode=FORCE_UNIFORM, force_uniform=(2e-6, 0.0, -1e-6))


@pytest.mark.parametrize("storage", ["f32", "f16s"])
@pytest.mark.parametrize("shape", [(40, 20, 8), (33, 17, 13), (64, 30, 29)])
def test_merged_z_chunks_equal_aa(gpu, shape, storage):
    """With fewer tiles than SMs the shadow-shell sweep splits z into chunks
    (one CTA per tile and chunk; the planes next to a chunk boundary come
    from a copy taken before the sweep).  The automatic chunk count, with a
    wall and a lid on the z faces."""
    import torch
    cfg = _zchunk_config(shape)
    f0 = start_state(cfg, seed=cfg.nz)
    ref = make_gpu(cfg, storage, "aa")
    load_state(ref, f0)
    ref.step(6)
    lat = make_gpu(cfg, storage, "merged")
    load_state(lat, f0)
    lat.step(6)
    assert torch.equal(_raw(lat), _raw(ref))


@pytest.mark.parametrize("storage", ["f32", "bf16s"])
@pytest.mark.parametrize("shape,nzc", [((64, 30, 29), 2), ((64, 30, 29), 3), ((64, 30, 29), 7),
                                       ((37, 19, 37), 2), ((37, 19, 37), 5), ((37, 19, 37), 9)])
def test_merged_explicit_z_chunks_equal_aa(gpu, monkeypatch, shape, nzc, storage):
    """Explicit chunk counts (LBM_MERGED_ZCHUNKS, read when the handle is
    created), uneven splits and the largest count nz // 4 included.  That the
    split is active is checked through the handle's size: it grows by the
    copy of the 2 (nzc - 1) planes next to the chunk boundaries."""
    import torch
    from paper_2208_05429_gb300 import lbm
    cfg = _zchunk_config(shape)
    nx, ny, nz = shape
    es = {"f32": 4, "bf16s": 2}[storage]
    monkeypatch.setenv("LBM_MERGED_ZCHUNKS", "1")
    one = lbm.lbm_required_bytes(lbm.make_config(shape, 0.7, cfg.bc, storage=storage, variant="merged"))
    monkeypatch.setenv("LBM_MERGED_ZCHUNKS", str(nzc))
    many = lbm.lbm_required_bytes(lbm.make_config(shape, 0.7, cfg.bc, storage=storage, variant="merged"))
    pitch = (nx + 15) // 16 * 16
    copy = 19 * 2 * (nzc - 1) * ny * pitch * es
    assert many - one == (copy + 255) // 256 * 256
    f0 = start_state(cfg, seed=nzc)
    lat = make_gpu(cfg, storage, "merged")
    load_state(lat, f0)
    lat.step(6)
    monkeypatch.delenv("LBM_MERGED_ZCHUNKS")
    ref = make_gpu(cfg, storage, "aa")
    load_state(ref, f0)
    ref.step(6)
    assert torch.equal(_raw(lat), _raw(ref))


def _walled_config(rng):
    """A random lattice with walls or lids on every face (the faces the
    neighbour-synchronised sweep serves), ragged against the 32-wide tiles
    and the 14-row bands."""
    import oracle
    from oracle import BC_LID, BC_WALL, FORCE_NONE, FORCE_UNIFORM
    nx, ny, nz = (int(v) for v in rng.integers([1, 1, 1], [100, 60, 12]))
    bc = tuple(BC_LID if rng.random() < 0.3 else BC_WALL for _ in range(6))
    lid = tuple(float(v) for v in rng.uniform(-0.04, 0.04, 3))
    fm = FORCE_UNIFORM if rng.random() < 0.5 else FORCE_NONE
    fu = tuple(float(v) for v in rng.uniform(-2e-5, 2e-5, 3)) if fm == FORCE_UNIFORM else (0.0, 0.0, 0.0)
    return oracle.Config(nx=nx, ny=ny, nz=nz, tau=float(rng.uniform(0.52, 1.2)), bc=bc, u_lid=lid,
                         force_mode=fm, force_uniform=fu)


@pytest.mark.parametrize("seed", range(16))
def test_neighbour_synchronised_sweep_equals_aa(gpu, monkeypatch, seed):
    """The neighbour-synchronised merged sweep (forced for every tile count
    with LBM_MERGED_SWEEP=neighbour) is bit-identical to AA on random walled
    lattices in the four formats that have it, over mixed step counts."""
    import torch
    from paper_2208_05429_gb300.lbm import lbm_required_bytes, make_config
    rng = np.random.default_rng(7000 + seed)
    cfg = _walled_config(rng)
    storage = ["f32", "f32s", "f16s", "bf16s"][seed % 4]
    f0 = start_state(cfg, seed=seed)
    monkeypatch.setenv("LBM_MERGED_SWEEP", "neighbour")
    shape = (cfg.nx, cfg.ny, cfg.nz)
    ns_bytes = lbm_required_bytes(make_config(shape, cfg.tau, cfg.bc, storage=storage, variant="merged"))
    lat = make_gpu(cfg, storage, "merged")
    monkeypatch.setenv("LBM_MERGED_SWEEP", "shadow")
    shadow_bytes = lbm_required_bytes(make_config(shape, cfg.tau, cfg.bc, storage=storage, variant="merged"))
    assert ns_bytes < shadow_bytes  # no shell shadow: the other sweep is not the one running
    monkeypatch.delenv("LBM_MERGED_SWEEP")
    load_state(lat, f0)
    for k in (2, 2, 1, 3, 2):
        lat.step(k)
    ref = make_gpu(cfg, storage, "aa")
    load_state(ref, f0)
    ref.step(10)
    assert torch.equal(_raw(lat), _raw(ref)), (cfg.nx, cfg.ny, cfg.nz, cfg.bc, storage)


def test_neighbour_synchronised_sweep_at_bench_size_equals_aa(gpu):
    """256^3 cavity, FP32: 152 tiles, one per SM, the sweep MERGED runs by
    default there; 6 steps equal AA bit for bit."""
    import torch
    import oracle
    cfg = oracle.cavity(256, 0.55)
    m = make_gpu(cfg, "f32", "merged")
    m.init_equilibrium()
    m.step(6)
    a = make_gpu(cfg, "f32", "aa")
    a.init_equilibrium()
    a.step(6)
    assert torch.equal(_raw(m), _raw(a))
