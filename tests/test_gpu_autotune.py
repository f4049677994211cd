"""The launch shape changes speed only: renders under different tile shapes,
CTA sizes, CTA counts and refill thresholds are bit-identical; the autotuner
returns a valid choice, caches it in memory and in a file, and leaves the
context on it."""
import json

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


SHAPES = [dict(tile_w=8, tile_h=4, block=256, ctas_per_sm=0, refill=16),
          dict(tile_w=32, tile_h=1, block=128, ctas_per_sm=1, refill=1),
          dict(tile_w=4, tile_h=8, block=64, ctas_per_sm=2, refill=32),
          dict(tile_w=16, tile_h=2, block=256, ctas_per_sm=0, refill=9)]


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_launch_shape_does_not_change_results(G, prec):
    sc = S.globule(800, 760, 16.0, seed=7)
    W, H = 101, 67
    cam = S.ortho_camera(sc, W, H, angle_deg=10.0)
    p = S.Params(ao_samples=8, seed=3, precision=prec, shadows=True)
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc, lam=4.0)
        frames = []
        for t in SHAPES:
            G.gbrt_set_tuning(r.ctx, **t)
            assert G.gbrt_get_tuning(r.ctx) == t
            frames.append(gpu_frame(G, r, scene, grid, cam, W, H, S.default_lights(), p))
        for f in frames[1:]:
            assert all(np.array_equal(a, b) for a, b in zip(frames[0], f))


def test_bad_tuning_rejected(G):
    with G.Renderer(0) as r:
        before = G.gbrt_get_tuning(r.ctx)
        for bad in (dict(tile_w=5, tile_h=5), dict(block=48), dict(block=512), dict(refill=0), dict(refill=33)):
            with pytest.raises(G.GbrtError):
                G.gbrt_set_tuning(r.ctx, **dict(before, **bad))
        assert G.gbrt_get_tuning(r.ctx) == before


def test_autotune_choice_and_cache(G, tmp_path):
    from paper_0801_1500_gb300 import autotune as AT
    sc = S.globule(300, 285, 10.0, seed=2)
    W, H = 64, 48
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=4, seed=0)
    cache = str(tmp_path / "tune.json")
    with G.Renderer(0) as r:
        best, sh, gh = AT.autotune(r, sc, cam, W, H, S.default_lights(), p, reps=1, cache_path=cache)
        assert not best["cached"] and best["lambda"] in AT.LAMBDAS and best["ms"] > 0
        assert best["trials"] == len(AT.LAMBDAS) + len(AT.REFILLS) + len(AT.TILES) + len(AT.BLOCKS)
        assert G.gbrt_get_tuning(r.ctx) == best["tuning"]
        assert G.gbrt_grid_info(gh)["dims"] == G.gbrt_grid_info(r.upload(sc, lam=best["lambda"])[1])["dims"]
        stored = json.load(open(cache))
        key = AT.cache_key(sc, W, H, p.ao_samples, p.precision)
        assert stored[key]["lambda"] == best["lambda"] and stored[key]["tuning"] == best["tuning"]
    with G.Renderer(0) as r:
        again, _, _ = AT.autotune(r, sc, cam, W, H, S.default_lights(), p, reps=1, cache_path=cache)
        assert again["cached"] and again["lambda"] == best["lambda"] and again["tuning"] == best["tuning"]
        assert G.gbrt_get_tuning(r.ctx) == best["tuning"]
