"""The replica path of bench.py with two ranks on the CPU (gloo): every rank times its own
evaluations, the job's time is the slowest rank's, and the whole-job throughput counts every
rank's units (weak scaling; independent problems need no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench._rank_env() == (rank, world, rank)
        seconds = [0.5, 0.8][rank]   # rank 1 is the slow replica
        value, slowest = bench._job_throughput(100, seconds, world, dist, "cpu")
        q.put((rank, value, slowest))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, slowest in got:
        assert slowest == 0.8
        assert value == pytest.approx(2 * 100 / 0.8)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._job_throughput(10, 2.0, 1, None, None) == (5.0, 2.0)
