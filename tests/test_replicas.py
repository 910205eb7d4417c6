"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks, each with its own sequence, reduce
their timed-region lengths to the slowest rank's and report the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.replica_throughput(10, world, m), bench.replica_seed(rank))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    out = tmp.Manager().dict()
    tmp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == out[1][1] == pytest.approx(10 * 2 / 0.150)
    assert out[0][2] != out[1][2]  # independent sequences


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(280, 1, 1000.0) == 280.0
