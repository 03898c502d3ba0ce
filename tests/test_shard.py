"""Partitioning of independent solves over ranks (the multi-GPU form of the batched sweep:
no collective on the data path, only host-side timing and result reductions), checked on
the CPU: the pure partition, and two gloo ranks that each take their share of the 256-problem
sweep and meet only in the host reductions the benchmark uses."""
import datetime
import os
import socket

import numpy as np
import pytest

from paper_2404_04507_gb300 import shard
from paper_2404_04507_gb300 import workloads as W


def _sweep_costs():
    _, _, _, kl = W.sweep_params(256, seed=4)
    return (2.0 * kl) ** 4


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_problem_once(world):
    costs = np.random.default_rng(world).uniform(0, 10, size=97)
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(costs.size))
    assert all(p == sorted(p) for p in parts)


@pytest.mark.parametrize("world", [2, 4, 8])
def test_sweep_partition_is_balanced(world):
    costs = _sweep_costs()
    ld = shard.loads(costs, shard.partition(costs, world))
    # longest processing time first: no rank exceeds the mean by more than one problem
    assert ld.max() <= costs.sum() / world + costs.max()
    assert np.isclose(ld.sum(), costs.sum())


def test_partition_rejects_bad_input():
    with pytest.raises(ValueError):
        shard.partition([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)
    with pytest.raises(ValueError):
        shard.shard([1.0, 2.0], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    costs = _sweep_costs()
    mine = shard.shard(costs, world, rank)
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    # the benchmark's max-over-ranks reduction of a per-rank time (here: the rank's load)
    load = torch.tensor([float(costs[mine].sum())], dtype=torch.float64)
    dist.all_reduce(load, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([len(mine), load.item()] + [i for p in everyone for i in p], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_sweep(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    costs = _sweep_costs()
    parts = shard.partition(costs, world)
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert int(got[0]) == len(parts[r])
        assert got[1] == shard.loads(costs, parts).max()
        union = got[2:].astype(int)
        assert sorted(union.tolist()) == list(range(256))       # disjoint and complete

