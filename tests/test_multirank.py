"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own
seeded mesh, combine their step times (max) and pair counts (sum) the way the
benchmark does under torchrun."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2103_16841_gb300 import inputs
    m = inputs.sphere_mesh(1, 4, 2.0, 0.2, seed=1 + rank)      # rank r assembles its own jittered mesh
    ms, pairs = bench.aggregate(10.0 + rank, 1000 * (rank + 1), "cpu")
    out[rank] = (ms, pairs, float(m.stv_t.sum()))
    tdist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0][:2] == (11.0, 3000.0) and out[1][:2] == (11.0, 3000.0)
    assert out[0][2] != out[1][2]          # different jitter per rank


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(5.0, 7, "cpu") == (5.0, 7.0)
