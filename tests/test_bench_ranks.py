"""The replica path of bench.py (N > 1 ranks, one independent solve each):
max time and summed DOFs over ranks, on CPU with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, n = bench.combine_ranks(10.0 + rank, 100 + rank, dist, device="cpu")
    q.put((rank, ms, n))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_combine_ranks_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, n in res:
        assert ms == 11.0 and n == 201.0


def test_combine_ranks_single_process():
    import bench
    assert bench.combine_ranks(3.5, 7) == (3.5, 7.0)
