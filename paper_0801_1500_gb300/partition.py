"""Splitting one frame over several GPUs (the paper's pixels-over-ranks
decomposition, Sec. 2), and the timing reduction of multi-rank runs.

Frames are independent, so multi-GPU runs render whole frames per rank
(weak scaling, no collective on the data path). When one frame is split,
rank r takes the row bands r, r + world, r + 2 world, ... (interleaved bands
even out the uneven density of a molecule); each band renders with its
whole-image coordinates (``gbrt_render_item.row_begin/row_end``), so the
union of the ranks' bands is exactly the one-GPU image, and one gather of
the bands assembles it.
"""
from __future__ import annotations

from typing import List, Tuple


def bands_for_rank(height: int, rank: int, world: int, band_rows: int = 32) -> List[Tuple[int, int]]:
    """Row bands [begin, end) of a `height`-row image owned by `rank`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    if height < 0 or band_rows < 1:
        raise ValueError("bad height or band size")
    n = (height + band_rows - 1) // band_rows
    return [(b * band_rows, min(height, (b + 1) * band_rows)) for b in range(rank, n, world)]


def max_over_ranks(seconds: float) -> float:
    """Slowest rank's time (torch.distributed initialised), else the value itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    backend = dist.get_backend()
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
