"""Multi-rank split of the sweep and surrogate runs, on CPU with the gloo
backend (world size 2): the ranks' shares are disjoint and cover every
point, costly points are spread over the ranks, and the timed region is the
slowest rank's."""
import os
import socket

import pytest

from paper_1401_6047_gb300 import shard


def test_split_single_rank_is_everything():
    assert shard.split(5, 0, 1) == [0, 1, 2, 3, 4]
    assert shard.split(4, 0, 1, cost=[1, 5, 3, 5]) == [1, 3, 2, 0]


def test_split_balances_cost():
    cost = [float(i % 17) ** 2 + 1 for i in range(1000)]
    parts = [shard.split(1000, r, 4, cost) for r in range(4)]
    assert sorted(i for p in parts for i in p) == list(range(1000))
    loads = [sum(cost[i] for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.02


def test_split_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.split(10, 2, 2)
    with pytest.raises(ValueError):
        shard.split(3, 0, 1, cost=[1, 2])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cost = [float((7 * i) % 11 + 1) for i in range(37)]
        mine = shard.split(37, rank, world, cost)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        slow = shard.slowest(1.5 + rank)
        out.put((rank, parts, slow))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_cover_all_points_and_agree_on_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, parts, slow in res:
        flat = sorted(i for part in parts for i in part)
        assert flat == list(range(37))
        assert not set(parts[0]) & set(parts[1])
        assert slow == 2.5
