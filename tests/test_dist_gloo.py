"""The N > 1 host path on CPU ranks (gloo, world size 2): sessions shard with no
overlap and nothing lost, and the timing reduction takes the max over ranks."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2503_23410_gb300.dist import max_over_ranks, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(list(range(64)), rank, world)
    elapsed = [1.0 + rank, 10.0 - rank]
    red = max_over_ranks(elapsed)
    dist.barrier()
    q.put((rank, mine, red))
    dist.destroy_process_group()


def test_shard_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        rank, mine, red = q.get(timeout=120)
        out[rank] = (mine, red)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = out[0][0], out[1][0]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
    assert out[0][1] == out[1][1] == [2.0, 10.0]


def test_shard_single_rank_and_errors():
    assert shard([1, 2, 3], 0, 1) == [1, 2, 3]
    with pytest.raises(ValueError):
        shard([1], 2, 2)
