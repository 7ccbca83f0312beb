"""Multi-GPU path of the benchmark (replicas): world size 2 over gloo on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, ev = bench.reduce_replicas(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, device="cpu")
    out[rank] = (ms, ev)
    dist.destroy_process_group()


def test_reduce_replicas_two_ranks():
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (15.0, 3000.0)


def test_reduce_replicas_single_process():
    import bench
    assert bench.reduce_replicas(3.0, 7.0) == (3.0, 7.0)
