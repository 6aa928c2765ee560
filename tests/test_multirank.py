"""Multi-GPU host logic on CPU: world_size-2 gloo ranks.

Series are independent, so ranks split a batch with no collective in the data path
(weak scaling: each rank searches its own share); the only collectives are the
timing barrier and the max-over-ranks of the step time.  These tests run that logic
as two gloo processes: the shards partition the series and balance the cost, and the
reduced step time is the slowest rank's."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2004_03701_gb300 as ffa
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, costs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = ffa.shard_series(costs, rank, world)
        # every rank's shard, gathered
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        # max over ranks of a per-rank step time (here: the rank's total cost)
        t = torch.tensor([sum(costs[i] for i in mine)], dtype=torch.float64)
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = torch.tensor([float(len(mine))], dtype=torch.float64)
        dist.all_reduce(total)
        q.put((rank, mine, shards, float(t.item()), int(total.item())))
    finally:
        dist.destroy_process_group()


def _run(world, costs):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_ranks_partition_and_balance():
    b = synth.batch_uneven(40, 2 ** 10, 2 ** 14, seed=5, threads=1)
    costs = [s.n for s in b.series]
    out = _run(2, costs)
    shards = out[0][2]
    assert out[1][2] == shards                      # every rank sees the same split
    assert [o[1] for o in out] == shards
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(costs)))          # a partition of the series
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(costs)    # greedy balance bound
    assert all(o[3] == max(loads) for o in out)     # max-over-ranks time
    assert all(o[4] == len(costs) for o in out)     # units summed over ranks


def test_shard_single_rank_and_errors():
    assert ffa.shard_series([3, 1, 2], 0, 1) == [0, 1, 2]
    assert ffa.shard_series([], 0, 2) == []
    with pytest.raises(ValueError):
        ffa.shard_series([1], 2, 2)
