"""Autotuner for the render launch shape and grid density.

Searches, by coordinate descent on measured device time:
  * grid density lambda (cells per object) -- rebuilds the grid;
  * the AO lane refill threshold (how empty a warp may get before its idle
    lanes take new shadow rays together);
  * the primary-ray tile shape (tile_w x tile_h = 32 pixels per warp);
  * threads per CTA of the persistent kernels.
Each candidate is timed over a few renders of a representative frame with
CUDA events (median). Results are cached per (scene digest, width, height,
samples, precision) in memory and, when a path is given, in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
from typing import Dict, Optional

import numpy as np

from . import gbrt as G

LAMBDAS = (1.0, 2.0, 4.0, 8.0, 16.0)
REFILLS = (8, 12, 16, 20, 24)
TILES = ((8, 4), (16, 2), (4, 8), (32, 1))
BLOCKS = (128, 256)

_memory_cache: Dict[str, dict] = {}


def scene_digest(scene) -> str:
    h = hashlib.sha1()
    for a in (scene.spheres, scene.cylinders, scene.color_idx, scene.palette):
        a = np.ascontiguousarray(a)
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()[:20]


def cache_key(scene, width, height, spp, precision) -> str:
    return f"{scene_digest(scene)}:{width}x{height}:spp{spp}:p{precision}"


def _load_file(path):
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def _time_frame(renderer, scene_h, grid_h, camera, width, height, lights, params, reps):
    """Median device time (ms) of the whole render over `reps` renders."""
    import torch
    dev = f"cuda:{renderer.device}"
    dtype = torch.float64 if params.precision == G.FP64 else torch.float32
    out = torch.empty((height, width, 3), dtype=dtype, device=dev)
    cam, li, pa = G.make_camera(camera), G.make_lights(lights), G.make_params(params)
    s = renderer.stream
    G.gbrt_render(renderer.ctx, scene_h, grid_h, cam, width, height, params.ao_samples, li, pa, out)
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        G.gbrt_render(renderer.ctx, scene_h, grid_h, cam, width, height, params.ao_samples, li, pa, out)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    G.gbrt_sync(renderer.ctx)
    return statistics.median(ts)


def autotune(renderer, scene, camera, width, height, lights, params, reps: int = 3,
             cache_path: Optional[str] = None, use_cache: bool = True, verbose: bool = False):
    """Tune for one frame shape. Returns (best dict, scene handle, grid handle).

    The returned handles are uploaded on `renderer` with the best lambda and
    the renderer's context is left on the best tuning.
    """
    key = cache_key(scene, width, height, params.ao_samples, params.precision)
    file_cache = _load_file(cache_path)
    hit = _memory_cache.get(key) or (file_cache.get(key) if use_cache else None)
    if use_cache and hit:
        t = dict(hit["tuning"])
        G.gbrt_set_tuning(renderer.ctx, **t)
        sh, gh = renderer.upload(scene, lam=hit["lambda"])
        return dict(hit, cached=True), sh, gh

    log = []
    base = G.gbrt_get_tuning(renderer.ctx)
    best = {"lambda": 2.0, "tuning": dict(base), "ms": float("inf")}

    # 1. grid density with the current launch shape
    handles = {}
    for lam in LAMBDAS:
        sh, gh = renderer.upload(scene, lam=lam)
        ms = _time_frame(renderer, sh, gh, camera, width, height, lights, params, reps)
        log.append(("lambda", lam, ms))
        handles[lam] = (sh, gh)
        if ms < best["ms"]:
            best.update(ms=ms, **{"lambda": lam})
    for lam, (sh, gh) in handles.items():
        if lam != best["lambda"]:
            renderer.free(sh, gh)
    sh, gh = handles[best["lambda"]]

    # 2. launch shape, one knob at a time
    def trial(**kw):
        t = dict(best["tuning"], **kw)
        G.gbrt_set_tuning(renderer.ctx, **t)
        ms = _time_frame(renderer, sh, gh, camera, width, height, lights, params, reps)
        log.append((kw, ms))
        if ms < best["ms"]:
            best.update(ms=ms, tuning=t)

    for rf in REFILLS:
        trial(refill=rf)
    for tw, th in TILES:
        trial(tile_w=tw, tile_h=th)
    for blk in BLOCKS:
        trial(block=blk)
    G.gbrt_set_tuning(renderer.ctx, **best["tuning"])
    best["trials"] = len(log)
    if verbose:
        for row in log:
            print("autotune", row)
    _memory_cache[key] = {k: best[k] for k in ("lambda", "tuning", "ms")}
    if cache_path:
        file_cache[key] = _memory_cache[key]
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(file_cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(best, cached=False), sh, gh
