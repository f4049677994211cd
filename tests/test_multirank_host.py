"""Multi-rank host logic on CPU with gloo (world size 2): the frame partition
covers every row exactly once, and the timing reduction takes the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_0801_1500_gb300 import partition as P


def test_bands_partition_exactly():
    for H in (1, 31, 32, 33, 1137, 4548):
        for world in (1, 2, 3, 8):
            rows = []
            for r in range(world):
                rows += [j for a, b in P.bands_for_rank(H, r, world, 32) for j in range(a, b)]
            assert sorted(rows) == list(range(H))
    with pytest.raises(ValueError):
        P.bands_for_rank(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank "renders" its bands; gather them and check the union
    mine = P.bands_for_rank(1137, rank, world, 32)
    allb = [None] * world
    dist.all_gather_object(allb, mine)
    rows = sorted(j for bands in allb for a, b in bands for j in range(a, b))
    t = P.max_over_ranks(0.5 + rank)
    q.put((rank, rows == list(range(1137)), t))
    dist.destroy_process_group()


def test_gloo_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(ok for _, ok, _ in res)
    assert all(t == 1.5 for _, _, t in res)
