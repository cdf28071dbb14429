"""Host logic of the multi-GPU benchmark (independent replicas, one per
rank): the timed region is the slowest rank's and the value is the
whole-job throughput.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [120.0, 150.0][rank]
    ms = bench.slowest_rank_ms(ms_local, True, "cpu")
    out[rank] = (ms, bench.whole_job_mlups(world, 256 ** 3, 100, ms))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    # 2 replicas x 256^3 cells x 200 time steps in 150 ms
    expect = 2 * 256 ** 3 * 200 / (150.0 * 1e3)
    assert out[0][1] == pytest.approx(expect) and out[1][1] == pytest.approx(expect)


def test_single_rank_value():
    import bench
    assert bench.slowest_rank_ms(10.0, False, "cpu") == 10.0
    assert bench.whole_job_mlups(1, 1000, 5, 1.0) == pytest.approx(1000 * 10 / 1e3)
