"""The multi-GPU bench path is replicas only: ranks run independent copies of
the workload and meet once, for the MAX of their timings.  Checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    elapsed = 100.0 + 50.0 * rank        # rank 1 is the slow one
    ms, value = bench.replica_aggregate(elapsed, 1e9, world, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replica_aggregate_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in out:
        assert ms == 150.0                          # the slowest rank's time
        assert abs(value - 2 * 1e9 / 0.150) < 1e-3  # units of both ranks over it


def test_replica_aggregate_single():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, value = bench.replica_aggregate(200.0, 1e9, 1, "cpu")
    assert ms == 200.0 and abs(value - 5e9) < 1e-6
