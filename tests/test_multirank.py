"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.

The benchmark runs one independent replica per rank ("replicas only": a single
case does not shard without a halo exchange), so the only cross-rank steps are
the barrier before the timed region and the maximum of the timed-region
lengths; the reported value is all ranks' particle-steps over that maximum.
"""
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


def _worker(rank, world, port, times, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t = bench.aggregate_time(times[rank], world)
    v = bench.job_value(1000, 10, t, world)
    out[rank] = (t, v)
    dist.destroy_process_group()


@pytest.mark.parametrize("times", [(12.5, 20.0), (30.0, 7.0)])
def test_two_ranks_report_the_slowest_time(times):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    tmax = max(times)
    for r in range(2):
        t, v = out[r]
        assert t == tmax
        assert abs(v - 2 * 1000 * 10 / (tmax * 1e-3)) < 1e-6 * v


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_time(3.5, 1) == 3.5
    assert bench.job_value(100, 4, 2.0, 1) == 100 * 4 / 2e-3
