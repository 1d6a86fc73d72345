"""Multi-process path of bench.py on CPU (gloo, world size 2).

The Ant System shards across GPUs only as independent replicas (instances
are independent; there is no data-path collective).  What the ranks share is
the timing protocol: a barrier around the timed region and the maximum of the
ranks' times, so the whole-job throughput is all units over the slowest
rank.  These tests run that protocol with the gloo backend.
"""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        slowest = bench.max_over_ranks(times[rank], world)
        value = bench.replica_throughput(1000.0, times[rank], world)
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.5, 2.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1000.0 / 2.0)


def _failing_worker(rank, world, port, out):
    import datetime
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    import bench
    if rank == 1:
        # this replica dies between steps, with nothing in flight
        os._exit(3)
    try:
        bench.barrier(world)
        out.put((rank, "passed"))
    except Exception as exc:  # the surviving rank learns of it on the host
        out.put((rank, type(exc).__name__))


def test_a_dead_replica_fails_the_barrier_instead_of_hanging():
    import multiprocessing as mp
    import time
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    rank, outcome = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and outcome != "passed"
    assert procs[1].exitcode == 3
    assert time.time() - t0 < 100


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(10.0, 2.0, 1) == 5.0
