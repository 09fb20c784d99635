"""Multi-GPU path of the benchmark on the CPU: one matrix per rank
(replicas, no collective on the data path); the job's rate is the sum of the
ranks' work over the slowest rank's time.  Two gloo ranks on 127.0.0.1."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [100.0, 250.0][rank]           # the second rank is slower
    flops_local = [2.0e12, 2.0e12][rank]
    ms, value = bench.replica_rate(ms_local, flops_local, world, torch.device("cpu"))
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replica_rate_two_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 250.0                            # the slowest rank's time
        assert value == pytest.approx(4.0e12 / 0.25 / 1e12)  # all ranks' work over it


def test_replica_rate_one_rank():
    sys.path.insert(0, ROOT)
    import bench

    ms, value = bench.replica_rate(50.0, 1.0e12, 1, None)
    assert ms == 50.0 and value == pytest.approx(20.0)
