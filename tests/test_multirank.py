"""The multi-rank path of bench.py (replicas: each rank runs its own
register, the job's time is the slowest rank's) with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]                       # rank 1 is the slow one
    t = bench.job_max(ms, world, "cpu")
    out[rank] = (t, bench.job_throughput(1259 * 3, world, t / 1e3))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    t, thr = out[0]
    assert t == 180.0
    assert thr == pytest.approx(1259 * 3 * 2 / 0.180)


def test_single_rank_is_identity():
    import bench
    assert bench.job_max(42.0, 1, "cpu") == 42.0
    assert bench.job_throughput(100, 1, 2.0) == 50.0
