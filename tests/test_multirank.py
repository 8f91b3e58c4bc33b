"""Multi-rank path of the benchmark on the CPU: two gloo ranks shard independent geometries
with no data-path collective and agree on the maximum of their timed regions."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2605_20918_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    steps = shard.rank_steps(rank, world, 5)
    geoms = [shard.geometry_of(s, 20) for s in steps]
    local_time = 1.0 + rank  # rank 1 is the slow one
    tmax = shard.max_over_ranks(local_time)
    out[rank] = (steps, geoms, tmax)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that already runs threads
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, g0, t0 = res[0]
    s1, g1, t1 = res[1]
    assert not set(s0) & set(s1)                      # disjoint work
    assert sorted(s0 + s1) == list(range(10))         # every step exactly once
    assert t0 == t1 == 2.0                            # max over ranks
    assert shard.seconds_per_build(t0, 5, world) == pytest.approx(0.2)


def test_single_process_helpers():
    assert shard.rank_steps(0, 1, 3) == [0, 1, 2]
    assert shard.geometry_of(23, 20) == 3
    assert shard.max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        shard.rank_steps(2, 2, 1)
