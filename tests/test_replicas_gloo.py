"""Multi-GPU path (replicas only) on CPU: two gloo ranks reduce their step times
with MAX and report the whole-job throughput exactly as bench.py does."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slowest
    v, ms = bench.replica_throughput(local_ms, iters=200, steps=5, world=world, device="cpu")
    out[rank] = (v, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        v, ms = out[rank]
        assert ms == 200.0
        assert abs(v - world * 200 * 5 / 0.2) < 1e-9


def test_replica_throughput_single_rank():
    import bench
    v, ms = bench.replica_throughput(50.0, iters=200, steps=5, world=1)
    assert ms == 50.0 and abs(v - 200 * 5 / 0.05) < 1e-9
