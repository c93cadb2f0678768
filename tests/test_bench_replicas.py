"""Multi-GPU is replicas only (each rank evaluates its own copy of the
workload, no collective on the data path); the job's throughput is the units
of all ranks over the slowest rank's time.  Checked with two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.004, 0.010][rank]                  # seconds per step on this rank
    t, value = bench.replica_throughput(local, 1.0e9, world, dist, torch.device("cpu"))
    out[rank] = (t, value)
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, value = res[r]
        assert t == pytest.approx(0.010)
        assert value == pytest.approx(world * 1.0e9 / 0.010)


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    t, value = bench.replica_throughput(0.5, 10.0, 1)
    assert (t, value) == (0.5, 20.0)
