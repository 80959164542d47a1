"""The multi-GPU path of bench.py is replicas only: each rank runs its own product and the job's
throughput is the units all ranks processed divided by the slowest rank's time.  This runs that
reduction on two CPU ranks (gloo), with unequal per-rank times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 10 (r + 1) ms for its step and 5 ms for the other one
        mx, rates = bench.replica_throughput([10.0 * (rank + 1), 5.0], 1e12, dist)
        out.put((rank, mx, rates))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rates in res:
        assert mx == [20.0, 5.0]                      # the slowest rank's times, on every rank
        assert rates[0] == pytest.approx(2e12 / 0.020)  # both ranks' units over the max time
        assert rates[1] == pytest.approx(2e12 / 0.005)


def test_replica_throughput_single_process():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    mx, rates = bench.replica_throughput([4.0], 8.0)
    assert mx == [4.0] and rates == [pytest.approx(2000.0)]
