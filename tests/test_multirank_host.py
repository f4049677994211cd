"""Multi-rank host logic on CPU with gloo (world size 2): the frame partition
covers every row exactly once and balances the paper frame's load, one gather
of the ranks' images assembles the one-rank image, and the timing reduction
takes the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_0801_1500_gb300 import partition as P
from paper_0801_1500_gb300 import scenes as S


def test_bands_partition_exactly():
    for H in (1, 31, 32, 33, 1137, 4548):
        for world in (1, 2, 3, 8):
            rows = []
            for r in range(world):
                rows += [j for a, b in P.bands_for_rank(H, r, world, 32) for j in range(a, b)]
            assert sorted(rows) == list(range(H))
    with pytest.raises(ValueError):
        P.bands_for_rank(10, 2, 2)


def test_bands_balance_the_paper_frame(oracle):
    # AO rays per rank (1 primary + 16 AO rays per hit pixel, hits from the
    # oracle's primary rays): interleaved 8-row bands within 1% of the mean at
    # 2, 4 and 8 ranks, and no worse than interleaved 32x32 tiles
    w = S.paper_1mp()
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, S.Params(ao_samples=0), mode="grid",
                        lam=2.0)
    load = 1 + 16 * (ref["id"] != oracle.MISS).reshape(w.height, w.width)
    H, W = load.shape
    for world in (2, 4, 8):
        per = [sum(load[a:b].sum() for a, b in P.bands_for_rank(H, r, world)) for r in range(world)]
        assert sum(per) == load.sum()
        bands = max(per) / np.mean(per)
        tiles = [0] * world
        k = 0
        for ty in range(0, H, 32):
            for tx in range(0, W, 32):
                tiles[k % world] += load[ty:ty + 32, tx:tx + 32].sum()
                k += 1
        assert bands <= 1.01 and bands <= max(tiles) / np.mean(tiles) + 1e-3, (world, bands)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _payload(H, W):
    """A per-pixel function of (i, j) standing in for a rendered image."""
    import torch
    j = torch.arange(H, dtype=torch.float64)[:, None]
    i = torch.arange(W, dtype=torch.float64)[None, :]
    img = torch.stack([torch.sin(0.37 * i + 0.11 * j), (i * 7919 + j * 104729) % 65521, i - j], dim=-1)
    return img.to(torch.float32)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    H, W = 1137, 97
    # each rank writes only its own bands of a whole-image buffer (the rest
    # stays NaN), then one all-gather of the buffers assembles the image
    full = _payload(H, W)
    mine = torch.full((H, W, 3), float("nan"), dtype=torch.float32)
    for a, b in P.bands_for_rank(H, rank, world):
        mine[a:b] = full[a:b]
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine)
    img = P.assemble(bufs, H)
    ok = bool(torch.equal(img, full))
    t = P.max_over_ranks(0.5 + rank)
    q.put((rank, ok, t))
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
