"""The multi-GPU path is replicas only (independent cities per rank, no
collective on the data path); its host logic — the job time is the slowest
rank's, the work the sum of the ranks' — checked with two gloo ranks on CPU."""
import os
import socket

import numpy as np
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


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2406_10661_gb300 import serving
    mine = serving.shard(list(range(64)), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = got
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_scenario_sharding_covers_every_scenario_once(world):
    """Batched/serving replicas: the ranks' shares are disjoint and together
    hold every scenario exactly once (no exchange is needed)."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        shares = res[r]
        flat = sorted(x for sh in shares for x in sh)
        assert flat == list(range(64))
        assert all(len(set(a) & set(b)) == 0 for i, a in enumerate(shares) for b in shares[i + 1:])


def test_shard_subset_generation_matches_full_set():
    """A rank that builds only its share gets the same scenarios as the full set."""
    from paper_2406_10661_gb300 import scenario as sc
    full = sc.batched_scenarios(6, n_hi=6000)
    part = sc.batched_scenarios(6, n_hi=6000, only=[1, 4])
    assert [p.name for p in part] == [full[1].name, full[4].name]
    for a, b in zip(part, [full[1], full[4]]):
        assert np.array_equal(a.veh.routes, b.veh.routes) and np.array_equal(a.veh.dep, b.veh.dep)
