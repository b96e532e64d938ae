"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
solves an independent instance, so the job reports the slowest rank's time
and the sum of all ranks' cell-updates; no collective touches the data."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    ms, upd = bench.reduce_over_ranks(dist, torch, 100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
    out[rank] = (ms, upd)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (150.0, 3000.0)
