"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timing
reduction is the maximum over ranks on every rank, and ranks draw distinct
inputs (weak scaling).  No GPU is involved."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        mine = [1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)]
        got = bench.reduce_max(mine, world)
        dist.barrier()
        q.put((rank, got, [bench.rank_seed(rank, li) for li in range(5)]))
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_rank_seeds_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, got, seeds in out:
        assert got == [2.0, 5.0, 0.5]
    assert set(out[0][2]).isdisjoint(out[1][2])


def test_reduce_max_single_rank_is_identity():
    import bench
    assert bench.reduce_max([3.0, 1.0], 1) == [3.0, 1.0]
