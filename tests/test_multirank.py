"""Host-side logic of the multi-rank benchmark path on CPU with the gloo
backend (world size 2): per-rank cells, sharding of independent work and the
max-over-ranks timing.  No GPU and no collective on the data path."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(bench.shard(13, rank, world))
        t = bench.max_over_ranks(1.5 + rank, device="cpu")
        q.put((rank, mine, t, bench.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(13))        # disjoint cover
    assert abs(len(shards[0]) - len(shards[1])) <= 1
    assert all(o[2] == 2.5 for o in out)                          # max over ranks
    assert out[0][3] != out[1][3]                                 # each rank its own cell


@pytest.mark.parametrize("n,w", [(0, 3), (5, 1), (7, 4), (96, 8)])
def test_shard_is_a_partition(n, w):
    parts = [list(bench.shard(n, r, w)) for r in range(w)]
    assert sum(parts, []) == list(range(n))
