"""The N > 1 host path of bench.py on CPU: world size 2 over gloo.

The product does not shard here (replicas only): every rank runs the whole
workload, the job time is the slowest rank's (an all-reduce MAX of the timed
totals) and the throughput counts the units of all ranks.  These tests run the
same helpers bench.py uses, in two gloo processes on 127.0.0.1.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 80.0][rank]          # a slow and a fast rank
    t_max = bench.max_over_ranks(local, dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, bench.job_throughput(1000, world, 10, t_max)))


def test_slowest_rank_sets_the_job_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [120.0, 120.0]
    # 2 ranks x 1000 units x 10 steps in 0.12 s
    assert out[0][2] == pytest.approx(2 * 1000 * 10 / 0.120)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.job_throughput(2 ** 20, 1, 10, 169.0) == pytest.approx(10 * 2 ** 20 / 0.169)


def _leaving_worker(rank, world, port, q):
    import datetime
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=15))
    import bench
    if rank == 1:
        # leaves between steps: joined the group, no collective of its own in flight
        q.put((rank, "left"))
        q.close()
        q.join_thread()          # the message is sent before the abrupt exit
        os._exit(3)
    try:
        bench.max_over_ranks(100.0, dist, torch.device("cpu"))
        q.put((rank, "no error"))
    except Exception:
        q.put((rank, "error"))


def test_lost_rank_fails_the_collective_instead_of_hanging():
    """A rank that exits between steps: the remaining rank's all-reduce of the
    timed totals raises (closed connection or the process-group timeout), so the
    job ends with an error instead of waiting forever."""
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert out == {0: "error", 1: "left"}
    assert procs[1].exitcode == 3
    assert time.time() - t0 < 110
