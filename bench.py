#!/usr/bin/env python3
"""Throughput of the D3Q19 hot path on GB300: MLUPS and the HBM roofline.

Workload (the benchmark configuration): lid-driven cavity 256^3, D3Q19 BGK,
tau = 0.55, lid u = (0.05, 0, 0) on the z+ face, half-way bounce-back on the
other five faces, fluid at rest at t = 0; FP32 storage and arithmetic; the
two-step merged sweep by default (on this lattice the neighbour-synchronised
kernel; --variant selects the single-copy AA pair or two lattices; the
other schedules, storage formats, collision models and the D3Q15 / D3Q27
lattices are reported under "variants", the shadow-shell merged sweep as
merged_shadow; --lattice 15 or 27 times one of those lattices instead, with
the single-step schedules).  One benchmark step = two lattice
time steps over all 16.8 M cells (one merged sweep, or an AA even/odd pair).
MLUPS counts every cell as a fluid node (million lattice-node updates per
second).

Three further modes print their own JSON line instead of the benchmark line:
``--sweep`` (cavity cubes 64^3 .. 768^3, FP32 and FP16-shifted storage, AA
and merged, plus the host oracle at 32^3, 64^3 and 128^3 on all host
threads and on one, and the paper's own CPU algorithms -- Alg. 1, Alg. 2
with and without prisms and its stride search, Alg. 3 on all host threads
-- at 64^3, 128^3 and 256^3),
``--precision-study`` (periodic Taylor-Green box 512^3, U0 = 0.04, tau =
0.52: FP32 / FP16 / BF16 storage against an FP64 run of the same case,
kinetic energy every 100 steps and max-norm velocity error) and
``--adjoint-study`` (the adjoint/forward time ratio on the differentiable
channel 128 x 64 x 64, the same figures as the benchmark line's "adjoint").

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs an
independent replica on its own GPU (the update shards only through a halo
exchange that this single-GPU build does not implement): value = the cells
all ranks updated / the slowest rank's time.

Besides the oracle's "cpu_baseline", the line carries "cpu_paper": the
paper's parallel two-step memory-aware LBM (Alg. 3, FP64, OpenMP on the host
cores, cpu_memaware) on the benchmark cavity itself, with its prism stride
chosen by the paper's stride search.

``--impl reference`` times the FP64 CPU oracle (the plain two-lattice
definition of the step, OpenMP on the host cores) on a bounded sample of the
same workload and prints the same line with ``"impl": "reference"``.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPS and % of HBM roofline per precision; adjoint/forward step ratio"
UNIT = "MLUPS"
TAU = 0.55
U_LID = (0.05, 0.0, 0.0)
FALLBACK_HBM_GBS = 6800.0
Q = 19
ELEM = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2, "bf16s": 2}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "f32s": "f32", "f16s": "f32 (f16 storage)", "bf16s": "f32 (bf16 storage)"}


def workload_name(n: int, q: int = Q) -> str:
    return (f"lid-driven cavity {n}^3, D3Q{q} BGK, tau={TAU}, lid u=(0.05,0,0) on z+, half-way bounce-back "
            f"on the other faces, initial rest state")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000, help="timed merged sweeps (2 time steps each)")
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=256)
    p.add_argument("--storage", default="f32", choices=sorted(ELEM))
    p.add_argument("--variant", default="merged", choices=["merged", "aa", "two_lattice"])
    p.add_argument("--lattice", type=int, default=Q, choices=[15, 19, 27],
                   help="velocity set of the timed leg (D3Q15 and D3Q27: single-step schedules)")
    p.add_argument("--no-extras", action="store_true", help="skip the per-variant, adjoint and CPU legs")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle baseline")
    p.add_argument("--sweep", action="store_true", help="cavity size sweep (prints its own JSON line)")
    p.add_argument("--sweep-sizes", default="64,128,256,512,768")
    p.add_argument("--precision-study", action="store_true", help="512^3 Taylor-Green precision study")
    p.add_argument("--study-size", type=int, default=512)
    p.add_argument("--study-steps", type=int, default=2000)
    p.add_argument("--adjoint-study", action="store_true",
                   help="adjoint/forward time ratio on the differentiable channel alone (prints its own JSON line)")
    return p.parse_args()


# ----------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


CSRC = os.path.join(ROOT, "paper_2208_05429_gb300", "csrc")


def source_closure(unit: str, read=None) -> list:
    """The csrc files a translation unit is compiled from: the unit and every
    header it includes with #include "...", transitively (sorted names).
    read(name) returns a file's text (default: the working tree)."""
    read = read or (lambda name: open(os.path.join(CSRC, name)).read())
    seen, todo = set(), [unit]
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.add(name)
        for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', read(name), re.M):
            if os.path.exists(os.path.join(CSRC, inc)):
                todo.append(inc)
    return sorted(seen)


def kernel_digest(unit: str, read=None) -> str:
    """Digest of the sources of one translation unit (names and contents):
    a kernel's recorded counters stay valid while these are unchanged."""
    read = read or (lambda name: open(os.path.join(CSRC, name)).read())
    h = hashlib.sha256()
    for name in source_closure(unit, read):
        h.update(name.encode())
        h.update(read(name).encode())
    return h.hexdigest()[:16]


def recorded_traffic(key: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        ent = d.get(key)
        if ent and ent.get("kernel_digest") == kernel_digest(ent["unit"]):
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        max_mhz = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * max_mhz] or rows
        reasons = set()
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names[1:], r[2][1:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max_mhz,
                "reasons": sorted(reasons), "samples": len(rows)}


def slowest_rank_ms(ms, dist_on, device):
    """The timed region's length on the slowest rank (max over ranks)."""
    if not dist_on:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells, steps, ms):
    """Whole-job throughput of `world` independent replicas, each running
    `steps` bench steps (two time steps each) of a `cells`-cell lattice in the
    slowest rank's `ms`."""
    return world * cells * 2 * steps / (ms * 1e3)


def sync_all(dist_on):
    import torch
    torch.cuda.synchronize()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
        torch.cuda.synchronize()


# ------------------------------------------------------------------ GPU legs

def make_cavity(n, storage, variant, collision="bgk", lattice=19):
    from paper_2208_05429_gb300.lbm import CAVITY_BC, Lattice
    return Lattice((n, n, n), TAU, bc=CAVITY_BC, u_lid=U_LID, storage=storage, variant=variant,
                   collision=collision, lattice=lattice)


def alg_bytes_per_launch(kernel: str, storage: str, cells: int, q: int = Q) -> float:
    """Algorithmic DRAM bytes of one launch: every population read and written
    once per round trip (a merged sweep is one round trip for two steps)."""
    return 2.0 * q * ELEM[storage] * cells


def time_variant(n, storage, variant, steps, warmup, dist_on=False, sweep_env=None, collision="bgk", lattice=19):
    """(elapsed ms over `steps` calls of step(2), per-kernel records, lattice).
    sweep_env: value of LBM_MERGED_SWEEP while the lattice is created (None:
    the library's own choice)."""
    import torch
    old = os.environ.get("LBM_MERGED_SWEEP")
    if sweep_env is not None:
        os.environ["LBM_MERGED_SWEEP"] = sweep_env
    try:
        lat = make_cavity(n, storage, variant, collision, lattice)
    finally:
        if sweep_env is not None:
            if old is None:
                del os.environ["LBM_MERGED_SWEEP"]
            else:
                os.environ["LBM_MERGED_SWEEP"] = old
    lat.init_equilibrium()
    for _ in range(warmup):
        lat.step(2)
    sync_all(dist_on)
    st = lat.stream
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    lat.profile(True)
    start.record(st)
    for _ in range(steps):
        lat.step(2)
    end.record(st)
    end.synchronize()
    lat.profile(False)
    sync_all(dist_on)
    return start.elapsed_time(end), lat.profile_read(), lat


def time_kstep(n, storage, K, sweeps, warmup):
    """(elapsed ms over `sweeps` calls of step(K), per-kernel records) of the
    K-step sweep on the cavity: one K-step sweep per call."""
    import torch
    from paper_2208_05429_gb300.lbm import CAVITY_BC, Lattice
    lat = Lattice((n, n, n), TAU, bc=CAVITY_BC, u_lid=U_LID, storage=storage, variant="kstep", sweep_steps=K)
    lat.init_equilibrium()
    for _ in range(warmup):
        lat.step(K)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    lat.profile(True)
    start.record(lat.stream)
    for _ in range(sweeps):
        lat.step(K)
    end.record(lat.stream)
    end.synchronize()
    lat.profile(False)
    prof = lat.profile_read()
    del lat
    return start.elapsed_time(end), prof


def roofline_of(prof, kernel, storage, cells, peak, peak_kind, q=Q):
    if kernel not in prof:
        return None
    launches, ms = prof[kernel]
    avg = ms / launches
    byts = alg_bytes_per_launch(kernel, storage, cells, q)
    achieved = byts / (avg * 1e-3) / 1e9
    traffic = recorded_traffic(f"{kernel}_{storage}_{round(cells ** (1 / 3))}" + ("" if q == Q else f"_d3q{q}"))
    return {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "alg_bytes_per_launch": byts, "avg_launch_ms": round(avg, 5), "launches": launches}


def e2e_leg(n, storage, variant, steps, warmup):
    """Same metric end to end through the public API with host buffers: the
    timed region uploads the initial populations from pinned host memory,
    runs the steps with an FP64 mass/momentum/energy read-back every 100 time
    steps, and downloads the final density and velocity fields."""
    import torch
    lat = make_cavity(n, storage, variant)
    lat.init_equilibrium()
    host_f = lat.populations(torch.float32).cpu().pin_memory()
    dev_f = torch.empty_like(host_f, device=lat.device)
    host_rho = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    host_u = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    every = 50
    for _ in range(warmup):
        lat.step(2)
    # the call pattern of the timed region once, so that its CUDA graph is
    # captured here and only replayed there
    lat.step(2 * min(every, steps))
    torch.cuda.synchronize()
    st = lat.stream
    reads = 0
    start = torch.cuda.Event(enable_timing=True)
    up = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        start.record(st)
        dev_f.copy_(host_f, non_blocking=True)
        up.record(st)
        lat.init_populations(dev_f)
        done = 0
        while done < steps:  # one step(n) call per reduction interval
            k = min(every, steps - done)
            lat.step(2 * k)
            done += k
            if k == every:
                lat.reduce()
                reads += 1
        rho, u = lat.moments(torch.float32)
        host_rho.copy_(rho, non_blocking=True)
        host_u.copy_(u, non_blocking=True)
        end.record(st)
    end.synchronize()
    ms = start.elapsed_time(end)
    up_ms = start.elapsed_time(up)
    cells = n ** 3
    h2d = host_f.numel() * 4
    d2h = (host_rho.numel() + host_u.numel()) * 4 + reads * 5 * 8
    return {"value": round(cells * 2 * steps / (ms * 1e3), 1), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / steps, 1), "d2h_bytes_per_step": round(d2h / steps, 1),
            "ms": round(ms, 3), "h2d_ms": round(up_ms, 3), "h2d_GBs": round(h2d / (up_ms * 1e6), 1),
            "what": "pinned host populations -> device, steps with an FP64 reduction read every 100 time "
                    "steps, final rho and u -> pinned host; bytes per step amortised over the run"}


def adjoint_leg():
    """Adjoint/forward time ratio on the differentiable channel workload
    (128 x 64 x 64, periodic x, walls y and z, tau 0.6, 200 steps,
    checkpoint every 20, per-cell force, FP32)."""
    import torch
    from paper_2208_05429_gb300 import inputs
    from paper_2208_05429_gb300.lbm import Lattice
    NX, NY, NZ, T, K = 128, 64, 64, 200, 20
    F = torch.tensor(inputs.channel_force(NX, NY, NZ), device="cuda")
    bc = ("periodic", "periodic", "wall", "wall", "wall", "wall")
    lat = Lattice((NX, NY, NZ), 0.6, bc=bc, storage="f32", variant="aa", force=F)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    st = lat.stream
    res = {}
    for rep in range(2):
        lat.init_equilibrium()
        ev[0].record(st)
        lat.step(T)
        ev[1].record(st)
        lat.init_equilibrium()
        ev[2].record(st)
        lat.adjoint_forward(T, K)
        ev[3].record(st)
        _, u = lat.moments(torch.float32)
        target = torch.tensor(inputs.parabolic_target(NY, NZ), device=u.device, dtype=torch.float32)
        g = torch.zeros_like(u)
        g[0, :, :, NX - 1] = 2.0 * (u[0, :, :, NX - 1] - target) / target.numel()
        ev[4].record(st)
        lat.adjoint_backward(g)
        ev[5].record(st)
        torch.cuda.synchronize()
        res = {"forward_ms": ev[0].elapsed_time(ev[1]), "checkpointed_forward_ms": ev[2].elapsed_time(ev[3]),
               "backward_ms": ev[4].elapsed_time(ev[5])}
    res = {k: round(v, 3) for k, v in res.items()}
    res["ratio"] = round(res["backward_ms"] / res["forward_ms"], 3)
    res["workload"] = "channel 128x64x64, 200 steps, checkpoint every 20, FP32; ratio = backward / plain forward"
    return res


# ------------------------------------------------------------------ CPU legs

def oracle_mlups(n, budget_s, pairs=None, nthreads=None):
    """Time the FP64 oracle (two lattices, OpenMP) on an n^3 cavity: runs
    `pairs` double steps, or as many as fit in budget_s (at least one), on
    nthreads host threads (default: as configured)."""
    import numpy as np
    import oracle
    if nthreads is not None:
        before = oracle.threads()
        oracle.threads(nthreads)
        try:
            return oracle_mlups(n, budget_s, pairs)
        finally:
            oracle.threads(before)
    cfg = oracle.cavity(n, TAU, u_lid=U_LID)
    f = oracle.init_equilibrium(cfg)
    g = np.empty_like(f)
    oracle.step(cfg, f)  # warm the library and the pages
    done = 0
    t0 = time.perf_counter()
    while True:
        oracle._load().orc_step(__import__("ctypes").byref(cfg._c()), oracle._ptr(f), oracle._ptr(g))
        oracle._load().orc_step(__import__("ctypes").byref(cfg._c()), oracle._ptr(g), oracle._ptr(f))
        done += 2
        el = time.perf_counter() - t0
        if pairs is not None:
            if done >= 2 * pairs:
                break
        elif el >= budget_s:
            break
    return n ** 3 * done / el / 1e6, done, el


def paper_cpu_mlups(n, alg, tile, nthreads, sweeps=1, cells=None):
    """Time the paper's own CPU algorithm `alg` (cpu_memaware: "fuse" Alg. 1,
    "two_step" Alg. 2, "omp" Alg. 3) on the n^3 cavity: `sweeps` two-step
    sweeps (two Alg. 1 steps for "fuse") from the rest state."""
    import numpy as np
    import cpu_memaware as cm
    cfg = cm.Config(n, n, n, TAU, u_lid=U_LID)
    if cells is None:
        _, w = cm.lattice()
        cells = np.ascontiguousarray(np.broadcast_to(w, (n, n, n, 19)).astype(np.float64))
    t0 = time.perf_counter()
    cm.run_cells(alg, cfg, cells, 2 * sweeps, tile, nthreads)
    el = time.perf_counter() - t0
    return n ** 3 * 2 * sweeps / el / 1e6, el, cells


def paper_cpu_leg(n, budget_s):
    """The paper's Alg. 3 (OpenMP two-step prism, FP64) on the host cores with
    its stride search (Sec. 5.2: strides 8 .. 448, plus no prisms), one sweep
    per stride after a warm-up sweep, then the best stride for about
    budget_s."""
    import cpu_memaware as cm
    cm.build()
    nt = omp_threads()
    rate, el, cells = paper_cpu_mlups(n, "omp", 0, nt)  # warm-up (pages, threads)
    search = {}
    for tile in [t for t in (8, 16, 32, 64, 128, 256, 448) if t <= n] + [0]:
        rate, el, cells = paper_cpu_mlups(n, "omp", tile, nt, cells=cells)
        search[str(tile) if tile else "none"] = round(rate, 2)
    best = max(search, key=search.get)
    tile = 0 if best == "none" else int(best)
    sweeps = max(1, int(budget_s / max(el, 1e-3)))
    rate, el, cells = paper_cpu_mlups(n, "omp", tile, nt, sweeps=sweeps, cells=cells)
    _, w = cm.lattice()
    mass = float(cells.sum())
    del cells
    return {"value": round(rate, 3), "unit": UNIT, "cores": nt,
            "kind": "the paper's Alg. 3 (parallel two-step memory-aware LBM, OpenMP, FP64)",
            "prism_stride": best, "stride_search_MLUPS": search,
            "sample": f"{2 * sweeps} time steps of the {n}^3 cavity itself ({el:.1f} s)",
            "mass_conserved": abs(mass - n ** 3) / n ** 3 < 1e-10}


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # pick the largest sample edge whose estimated run fits ~2 minutes
    total_pairs = args.steps + args.warmup
    edge = 32
    for cand in (args.size, 192, 128, 96, 64, 48, 32):
        if cand > args.size:
            continue
        rate, _, _ = oracle_mlups(cand, 0.0, pairs=1)
        est = 2 * total_pairs * cand ** 3 / (rate * 1e6)
        if est <= 120.0:
            edge = cand
            break
    oracle_mlups(edge, 0.0, pairs=max(args.warmup, 0) or 1)
    rate, done, el = oracle_mlups(edge, 0.0, pairs=args.steps)
    cores = omp_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(rate, 3), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.size), "sample": f"{edge}^3 cavity of the same setup",
                   "time_steps_per_step": 2},
        "cpu_baseline": {"value": round(rate, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} time steps of a {edge}^3 cavity (same tau, lid and walls), "
                                   f"FP64 two-lattice oracle, OpenMP {cores} threads"},
        "e2e": {"value": round(rate, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main

def sweep(args):
    """Cavity size sweep: MLUPS and fraction of the measured HBM peak per
    size, storage and schedule (about 500 time steps each, at least ~1 s),
    and the host oracle at 32^3, 64^3 and 128^3 on all host threads and on one."""
    import torch
    from paper_2208_05429_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    peak, peak_kind = measured_peaks()
    rows = []
    for n in [int(v) for v in args.sweep_sizes.split(",")]:
        cells = n ** 3
        for st in ("f32", "f16s"):
            for var in ("aa", "merged"):
                steps = max(64, min(2000, int(4e10 / (cells * 2))))  # ~0.5-1 s at 40-60k MLUPS
                try:
                    # kernel fraction from a short profiled run (one launch per call) ...
                    _, prof, lat = time_variant(n, st, var, 5, 3)
                    # ... and MLUPS from one step(n) call, which replays captured CUDA graphs
                    lat.step(64)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(lat.stream)
                    lat.step(2 * steps)
                    e1.record(lat.stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    ok = abs(lat.reduce()[0] - cells) / cells < 1e-4
                    del lat
                    torch.cuda.empty_cache()
                except Exception as e:  # e.g. out of memory at the largest sizes
                    rows.append({"n": n, "storage": st, "variant": var, "error": repr(e)[:200]})
                    continue
                dk = {"merged": "merged", "aa": "aa_odd"}[var]
                r = roofline_of(prof, dk, st, cells, peak, peak_kind)
                rows.append({"n": n, "storage": st, "variant": var, "time_steps": 2 * steps,
                             "MLUPS": round(cells * 2 * steps / (ms * 1e3), 1),
                             "kernel": dk, "kernel_frac_of_peak": r["frac"] if r else None,
                             "kernel_GBs_alg": r["achieved"] if r else None, "mass_conserved": bool(ok)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    import oracle
    oracle.build()
    cpu = []
    for n in (32, 64, 128):
        for nt in (omp_threads(), 1):
            rate, done, el = oracle_mlups(n, 5.0, nthreads=nt)
            cpu.append({"n": n, "MLUPS": round(rate, 2), "time_steps": done, "seconds": round(el, 2),
                        "threads": nt, "nproc": os.cpu_count()})
    # the paper's four sequential solvers (Sec. 5.2: fuse, fuse prism -- not
    # built, Palabos's own --, 2-step, 2-step prism with its stride search)
    # and its parallel one (Alg. 3, all threads), FP64
    import cpu_memaware as cm
    cm.build()
    paper = []
    for n in (64, 128, 256):
        seq = {"fuse": round(paper_cpu_mlups(n, "fuse", 0, 1)[0], 2),
               "two_step": round(paper_cpu_mlups(n, "two_step", 0, 1)[0], 2)}
        tiles = [t for t in (8, 16, 32, 64, 128, 256) if t <= n]
        if n <= 128:
            seq["two_step_prism"] = {str(t): round(paper_cpu_mlups(n, "two_step", t, 1)[0], 2) for t in tiles}
        par = {str(t): round(paper_cpu_mlups(n, "omp", t, omp_threads())[0], 2) for t in tiles + [0]}
        paper.append({"n": n, "sequential_MLUPS": seq, "omp_MLUPS_by_stride": par, "threads": omp_threads()})
        print(json.dumps(paper[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "sweep", "workload": "lid-driven cavity n^3, tau 0.55, lid (0.05,0,0)",
                      "peak_GBs": peak, "peak_source": peak_kind, "gpu": rows, "cpu_oracle": cpu,
                      "cpu_paper_algorithms": paper}), flush=True)
    return 0


def precision_study(args):
    """Periodic Taylor-Green box: each storage format against an FP64 run of
    the same case (AA schedule, FP32 arithmetic for the 4- and 2-byte formats)."""
    import numpy as np
    import torch
    from paper_2208_05429_gb300 import build, inputs
    from paper_2208_05429_gb300.lbm import Lattice
    build.build()
    torch.cuda.set_device(0)
    n, steps, tau, U0 = args.study_size, args.study_steps, 0.52, 0.04
    u0 = torch.tensor(inputs.taylor_green_velocity(n, n, n, U0), dtype=torch.float32, device="cuda")
    every = 100

    def run(storage):
        lat = Lattice((n, n, n), tau, storage=storage, variant="aa")
        lat.init_equilibrium(None, u0)
        ke = []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for t in range(0, steps, every):
            ev0.record(lat.stream)
            lat.step(min(every, steps - t))
            ev1.record(lat.stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            ke.append(lat.reduce()[4])
        _, u = lat.moments(torch.float64 if storage == "f64" else torch.float32)
        del lat
        torch.cuda.empty_cache()
        return u, np.array(ke), ms

    u_ref, ke_ref, ms_ref = run("f64")
    umax = float(u_ref.abs().max())
    out = {"f64": {"MLUPS": round(n ** 3 * steps / (ms_ref * 1e3), 1), "KE_final": float(ke_ref[-1])}}
    for st in ("f32", "f16s", "bf16s"):
        u, ke, ms = run(st)
        err = float((u.double() - u_ref).abs().max()) / umax
        out[st] = {"MLUPS": round(n ** 3 * steps / (ms * 1e3), 1), "u_maxnorm_rel_err": err,
                   "KE_rel_err_final": float(abs(ke[-1] - ke_ref[-1]) / ke_ref[-1]),
                   "KE_rel_err_max": float(np.max(np.abs(ke - ke_ref) / ke_ref))}
        del u
        torch.cuda.empty_cache()
    out["speedup_f16s_vs_f32"] = round(out["f16s"]["MLUPS"] / out["f32"]["MLUPS"], 3)
    out["speedup_bf16s_vs_f32"] = round(out["bf16s"]["MLUPS"] / out["f32"]["MLUPS"], 3)
    print(json.dumps({"mode": "precision_study",
                      "workload": f"periodic Taylor-Green {n}^3, U0 {U0}, tau {tau}, {steps} steps, AA schedule",
                      "KE_every": every, "KE_f64": [float(v) for v in ke_ref], "results": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return sweep(args)
    if args.precision_study:
        return precision_study(args)
    if args.adjoint_study:
        import torch
        from paper_2208_05429_gb300 import build
        torch.cuda.set_device(0)
        build.build()
        print(json.dumps({"mode": "adjoint_study", **adjoint_leg()}))
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)

    from paper_2208_05429_gb300 import build
    if rank == 0 or not dist_on:
        build.build()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()

    n = args.size
    cells = n ** 3
    peak, peak_kind = measured_peaks()

    sampler = ClockSampler(local)
    sampler.start()
    ms, prof, lat = time_variant(n, args.storage, args.variant, args.steps, args.warmup, dist_on,
                                 lattice=args.lattice)
    clocks = sampler.stop()
    ms = slowest_rank_ms(ms, dist_on, "cuda")
    # mass check of the timed state: a broken kernel shows up here
    mass = lat.reduce()[0]
    ok = abs(mass - cells) / cells < 1e-5
    del lat

    value = whole_job_mlups(world, cells, args.steps, ms)
    dominant = {"merged": "merged", "aa": "aa_odd"}.get(args.variant, "two_lattice")
    if args.lattice != Q and dominant == "merged":
        dominant = "aa_odd"   # MERGED runs the AA pair on D3Q15 / D3Q27
    roof = roofline_of(prof, dominant, args.storage, cells, peak, peak_kind, args.lattice)
    launches = sum(v[0] for v in prof.values())
    if "snapshot" in prof and roof is not None:
        sn, sms = prof["snapshot"]
        mn, mms = prof["merged"]
        roof["snapshot_avg_launch_ms"] = round(sms / sn, 5)
        roof["step_frac_of_peak_alg"] = round(alg_bytes_per_launch("merged", args.storage, cells) /
                                              ((sms + mms) / mn * 1e-3) / 1e9 / peak, 4)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.storage], "data": "synthetic",
        "config": {"workload": workload_name(n, args.lattice), "cells": cells, "time_steps_per_step": 2,
                   "storage": args.storage, "variant": args.variant,
                   "l2": "no flush: the populations (%.2f GB) are larger than the 129 MB L2" %
                         (args.lattice * ELEM[args.storage] * cells / 1e9),
                   "parallelism": "independent replicas, one per GPU" if dist_on else "single GPU"},
        "roofline": roof, "gpu_launches": launches, "clocks": clocks, "mass_conserved": bool(ok),
    }

    if rank == 0 and not args.no_extras:
        try:
            line["e2e"] = e2e_leg(n, args.storage, args.variant, min(args.steps, 1000), 3)
        except Exception as e:  # keep the main line if a secondary leg fails
            line["e2e"] = {"error": repr(e)}
        variants = {}
        for st, var, env in (("f32", "merged", None), ("f32", "aa", None), ("f32", "two_lattice", None),
                             ("f32", "merged", "shadow"), ("f32s", "merged", None),
                             ("f16s", "merged", None), ("f16s", "aa", None), ("bf16s", "merged", None),
                             ("bf16s", "aa", None), ("f64", "aa", None), ("f32", "aa", "trt"),
                             ("f16s", "aa", "trt"), ("f32", "aa", "reg"), ("f16s", "aa", "reg"),
                             ("f32", "merged", "trt"), ("f32", "merged", "reg"), ("f32", "aa", "mrt"),
                             ("f32", "merged", "mrt"), ("f32", "aa", "d3q15"), ("f32", "aa", "d3q27"),
                             ("f16s", "aa", "d3q27"), ("f32", "two_lattice", "d3q27")):
            if (st, var, env) == (args.storage, args.variant, None):
                continue
            k = min(args.steps, 300)
            coll = env if env in ("trt", "reg", "mrt") else "bgk"
            q = int(env[3:]) if env and env.startswith("d3q") else Q
            vms, vprof, vl = time_variant(n, st, var, k, 5, sweep_env=env if env == "shadow" else None,
                                          collision=coll, lattice=q)
            del vl
            dk = {"merged": "merged", "aa": "aa_odd"}.get(var, "two_lattice")
            r = roofline_of(vprof, dk, st, cells, peak, peak_kind, q)
            name = f"{var}_{env}_{st}" if env else f"{var}_{st}"
            variants[name] = {"MLUPS": round(cells * 2 * k / (vms * 1e3), 1),
                              "kernel_frac_of_peak": r["frac"] if r else None,
                              "kernel": dk}
        for st, K in (("f32", 3), ("f32", 4), ("f16s", 3)):
            k = min(args.steps, 30)
            vms, vprof = time_kstep(n, st, K, k, 3)
            r = roofline_of(vprof, "kstep", st, cells, peak, peak_kind)
            variants[f"kstep{K}_{st}"] = {"MLUPS": round(cells * K * k / (vms * 1e3), 1),
                                          "kernel_frac_of_peak": r["frac"] if r else None, "kernel": "kstep"}
        line["variants"] = variants
        try:
            line["adjoint"] = adjoint_leg()
        except Exception as e:
            line["adjoint"] = {"error": repr(e)}
        if not dist_on:
            import oracle
            oracle.build()
            rate, done, el = oracle_mlups(n, args.cpu_seconds)
            line["cpu_baseline"] = {
                "value": round(rate, 3), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                "sample": f"{done} time steps of the {n}^3 cavity itself, FP64 two-lattice oracle "
                          f"({el:.1f} s, OpenMP)"}
            try:
                line["cpu_paper"] = paper_cpu_leg(n, 3.0)
            except Exception as e:
                line["cpu_paper"] = {"error": repr(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist_on:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
