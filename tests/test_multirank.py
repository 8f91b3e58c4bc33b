"""Multi-rank paths on the CPU with two gloo ranks: the benchmark's sharding of independent
geometries (no data-path collective; the ranks agree on the maximum of their timed regions),
and the colour-partitioned decomposition of one system (colours dealt to ranks, one
all-gather of the Ritz pairs before mu, each rank extracting the columns of its colours),
which must reproduce the single-process density matrix bit for bit."""
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


def _colour_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_2605_20918_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.water_box(125)
    H = synth.hamiltonian(g, "minimal")
    col, nc = oracle.color(g.pos, g.box, 8.0, 1004)
    sgn = oracle.probes(col, H.b, 1005)
    ne = synth.n_electrons(125)
    mine = shard.colour_partition(np.bincount(col, minlength=nc), world)[rank]
    # this rank's block-Lanczos problems only; the one exchange is the Ritz pairs
    ritz = oracle.ritz(H, col, sgn, nc, 10, colours=mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, [(c, ritz[c][0], ritz[c][1]) for c in mine])
    lists = sorted((x for part in gathered for x in part), key=lambda x: x[0])
    mu = oracle.solve_mu([(lam, w) for _, lam, w in lists], 0.05, ne)
    # the columns of this rank's colours, unsymmetrised; the gatherer adds and symmetrises them
    Pmine = oracle.density(H, col, sgn, nc, mu=mu, kT=0.05, solve_mu=False, m=10, flags=0, colour_subset=mine)["P"]
    parts = [None] * world
    dist.all_gather_object(parts, Pmine)
    if rank == 0:
        out["mu"] = mu
        out["P"] = sum(parts[1:], parts[0])
        out["colours"] = [x[0] for x in lists]
    out[f"mine{rank}"] = mine
    dist.destroy_process_group()


def test_colour_partition_deals_every_colour_once():
    sizes = [5, 9, 1, 7, 7, 3, 8]
    parts = shard.colour_partition(sizes, 3)
    assert sorted(c for p in parts for c in p) == list(range(len(sizes)))
    loads = [sum(sizes[c] for c in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert shard.colour_partition(sizes, 1) == [list(range(len(sizes)))]
    assert shard.colour_partition([4, 4], 3) == [[0], [1], []]


def test_colour_partitioned_density_on_two_gloo_ranks(oracle_lib):
    import numpy as np

    from paper_2605_20918_gb300 import synth
    from tests.dense_truth import symmetrize
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_colour_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    g = synth.water_box(125)
    H = synth.hamiltonian(g, "minimal")
    col, nc = oracle_lib.color(g.pos, g.box, 8.0, 1004)
    sgn = oracle_lib.probes(col, H.b, 1005)
    ref = oracle_lib.density(H, col, sgn, nc, kT=0.05, n_elec=synth.n_electrons(125), m=10)
    assert res["colours"] == list(range(nc))
    assert not set(res["mine0"]) & set(res["mine1"]) and res["mine0"] and res["mine1"]
    assert res["mu"] == ref["mu"]
    assert np.array_equal(symmetrize(H, res["P"]), ref["P"])
