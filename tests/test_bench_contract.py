"""The benchmark's reference arm on the host (no GPU): one JSON line with the
contract's keys, consistent values, and silence on every rank but 0 when
launched as several ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3", "--size", "32"]


def _run(cmd, extra_env=None):
    env = dict(os.environ, OMP_NUM_THREADS="2", MASTER_ADDR="127.0.0.1")
    env.update(extra_env or {})
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_line():
    lines = _run([sys.executable, *ARGS])
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and "32^3" in d["config"]["sample"]


def test_reference_arm_other_ranks_print_nothing():
    assert _run([sys.executable, *ARGS], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_reference_arm_under_torchrun_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), *ARGS, "--gpus", "2"]
    lines = _run(cmd)
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2


def test_recorded_traffic_is_keyed_to_each_kernels_sources():
    """Each recorded ncu figure names the translation unit its kernel is built
    from; the digest covers that unit and the headers it includes (so a new
    kernel elsewhere leaves it valid, an edit of those sources voids it)."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)
    assert rec
    for key, ent in rec.items():
        assert os.path.exists(os.path.join(bench.CSRC, ent["unit"])), key
        fresh = bench.kernel_digest(ent["unit"]) == ent["kernel_digest"]
        assert bench.recorded_traffic(key) == (ent["dram_bytes_per_launch"] if fresh else None), key
    closure = bench.source_closure("inst_f32.cu")
    assert {"inst_f32.cu", "launch.cuh", "nsweep.cuh", "kernels.cuh", "d3q19.cuh", "ops.h"} <= set(closure)
    assert "ksweep.cuh" not in closure and "dqn.cuh" not in closure
    files = {n: open(os.path.join(bench.CSRC, n)).read() for n in closure}
    base = bench.kernel_digest("inst_f32.cu", lambda n: files[n])
    edited = dict(files, **{"nsweep.cuh": files["nsweep.cuh"] + "\n// edit\n"})
    assert bench.kernel_digest("inst_f32.cu", lambda n: edited[n]) != base
