"""The multi-GPU path is replicas only (independent cities per rank, no
collective on the data path); its host logic — the job time is the slowest
rank's, the work the sum of the ranks' — checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.reduce_ranks(dist, dev_s=1.0 + rank, updates=1000.0 * (rank + 1))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_ranks_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        t, u = res[r]
        assert t == 2.0 and u == 3000.0  # max time, summed updates -> value = 1500 /s
