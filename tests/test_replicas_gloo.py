"""The N>1 path of bench.py runs independent replicas (one per GPU, no data
exchange): only the timing is reduced, max over ranks, and the job's
throughput is world x units / that time.  Checked here with two gloo ranks
on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [10.0, 25.0][rank]               # rank 1 is the slower replica
        t, v = bench.replica_throughput(local_ms, 5.0e11, world, torch.device("cpu"))
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 25.0
        assert v == pytest.approx(2 * 5.0e11 / 0.025 / 1e9)


def test_replica_throughput_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.replica_throughput(20.0, 1.0e12, 1, None)
    assert t == 20.0 and v == pytest.approx(1.0e12 / 0.02 / 1e9)
