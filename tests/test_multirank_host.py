"""Two-rank (gloo, CPU) checks of the multi-GPU host logic: every rank
computes the same cost-balanced split of a batch without communicating, the
split is disjoint and complete, and the step time is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2502_06377_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard.shard_by_cost(sizes, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = shard.max_over_ranks(1.0 + rank)
    out.put((rank, gathered, t))
    dist.destroy_process_group()


def test_two_rank_split_and_max_time():
    import numpy as np
    rng = np.random.default_rng(4)
    sizes = [int(v) for v in 64 * rng.integers(1, 17, size=512)]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in res:
        assert t == 2.0                       # max over ranks of 1.0, 2.0
        a, b = gathered
        assert sorted(a + b) == list(range(len(sizes)))
        assert not set(a) & set(b)
        la = sum(shard.cost(sizes[i]) for i in a)
        lb = sum(shard.cost(sizes[i]) for i in b)
        assert max(la, lb) / min(la, lb) < 1.01
    assert res[0][1] == res[1][1]


def test_split_is_deterministic_and_single_rank_identity():
    sizes = [100, 2000, 64, 512, 512, 4096]
    assert shard.shard_by_cost(sizes, 1, 0) == list(range(len(sizes)))
    assert shard.shard_by_cost(sizes, 3, 1) == shard.shard_by_cost(sizes, 3, 1)
    with pytest.raises(ValueError):
        shard.shard_by_cost(sizes, 2, 2)


@pytest.mark.parametrize("world", [2, 3, 4, 5, 8])
def test_split_partitions_and_respects_the_greedy_bound(world):
    """Every index on exactly one rank, and with many items of a few sizes the
    greedy split's largest load is within 2% of the lower bound
    max(total / world, largest item) on the optimum."""
    import numpy as np
    rng = np.random.default_rng(world)
    sizes = [int(v) for v in 64 * rng.integers(1, 17, size=300)]
    parts = [shard.shard_by_cost(sizes, world, r) for r in range(world)]
    flat = sorted(i for part in parts for i in part)
    assert flat == list(range(len(sizes)))
    loads = [sum(shard.cost(sizes[i]) for i in part) for part in parts]
    opt_lb = max(sum(loads) / world, max(shard.cost(s) for s in sizes))
    assert max(loads) <= 1.02 * opt_lb
