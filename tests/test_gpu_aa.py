"""GPU parity of supersampling (camera.aa = m: m x m regular sub-pixel grid,
box-filtered) against the FP64 oracle, through the C ABI.

The device reports hit ids and AO counts per sub-sample in the m-times finer
raster ([m H][m W]); the oracle lists them per pixel, sub-row, sub-column.
Colours are per pixel. The parity rule is the one of the plain render (hit
ids exact off grazing sub-samples, |dRGB| <= 1/255 on 99.9% of pixels, MAE
<= 1e-4).
"""
import dataclasses

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import assert_ids, assert_rgb, id_stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


@pytest.fixture(scope="module")
def R(G):
    r = G.Renderer(0)
    yield r
    r.close()


@pytest.fixture(scope="module")
def paper():
    return S.paper_scene()


def with_aa(cam, m):
    return dataclasses.replace(cam, aa=m)


def fine_to_oracle(fine, W, m, pixels):
    """Finer-raster array [m H][m W] -> oracle order [k m^2 + b m + a] over `pixels`."""
    fine = np.asarray(fine).reshape(-1, m * W)
    out = np.empty(len(pixels) * m * m, fine.dtype)
    for k, q in enumerate(pixels):
        i, j = q % W, q // W
        out[k * m * m:(k + 1) * m * m] = fine[m * j:m * j + m, m * i:m * i + m].ravel()
    return out


def render_aa(G, R, scene, grid, cam, W, H, lights, p):
    rgb, ids, vis = R.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
    G.gbrt_sync(R.ctx)
    return (rgb.cpu().numpy().reshape(-1, 3).astype(np.float64), ids.cpu().numpy().view(np.uint32),
            vis.cpu().numpy().view(np.uint32))


def check(rgb, ids, vis, ref, W, m, pixels, where):
    ids_o = fine_to_oracle(ids, W, m, pixels)
    vis_o = fine_to_oracle(vis, W, m, pixels)
    assert_ids(*id_stats(ids_o, ref), len(ids_o), where)
    assert_rgb(np.abs(rgb[pixels] - ref["rgb"]), where)
    return float((vis_o == ref["vis"].astype(np.uint32)).mean())


@pytest.mark.parametrize("prec", [S.PRECISION_FP64, S.PRECISION_FP32])
@pytest.mark.parametrize("m", [2, 3])
@pytest.mark.parametrize("kind", ["ortho", "pinhole"])
def test_supersampled_small_frame(G, R, oracle, prec, m, kind):
    sc = S.globule(2000, 1900, 25.0, seed=0)
    W, H = 97, 61   # ragged against the 8 x 4 primary tiles at every m
    cam = S.ortho_camera(sc, W, H, angle_deg=15.0) if kind == "ortho" else S.pinhole_camera(sc, W, H, angle_deg=40.0)
    cam = with_aa(cam, m)
    lights = S.default_lights()
    p = S.Params(ao_samples=6, seed=4, frame=2, precision=prec)
    scene, grid = R.upload(sc, lam=2.0)
    rgb, ids, vis = render_aa(G, R, scene, grid, cam, W, H, lights, p)
    assert ids.shape == (m * H, m * W)
    ref = oracle.render(sc, cam, W, H, lights, p, mode="grid", lam=2.0)
    vis_eq = check(rgb, ids, vis, ref, W, m, np.arange(W * H), f"m={m} {kind}")
    assert vis_eq >= (0.9999 if prec == S.PRECISION_FP64 else 0.999)
    R.free(scene, grid)


def test_supersampled_pinhole_paper_scene_sampled(G, R, oracle, paper):
    # 26,318 objects, 965 x 1137 pinhole view, 2 x 2 sub-samples, 16 AO samples, FP32 path
    W, H, m = 965, 1137, 2
    cam = S.pinhole_camera(paper, W, H, fov_deg=30.0, aa=m)
    lights = S.default_lights()
    p = S.Params(ao_samples=16, seed=0)
    scene, grid = R.upload(paper, lam=8.0)
    rgb, ids, vis = render_aa(G, R, scene, grid, cam, W, H, lights, p)
    rng = np.random.default_rng(11)
    pixels = np.sort(rng.choice(W * H, 3000, replace=False))
    ref = oracle.render(paper, cam, W, H, lights, p, pixels=pixels, mode="grid", lam=2.0)
    vis_eq = check(rgb, ids, vis, ref, W, m, pixels, "paper pinhole 2x2")
    assert vis_eq >= 0.999
    hit = ref["id"] != 0xFFFFFFFF
    assert 0.2 < hit.mean() < 0.95
    R.free(scene, grid)


def test_aa_one_is_the_plain_render(G, R):
    sc = S.globule(300, 285, 10.0, seed=9)
    W, H = 70, 50
    cam = S.ortho_camera(sc, W, H)
    scene, grid = R.upload(sc)
    p = S.Params(ao_samples=6, seed=2)
    a = render_aa(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    b = render_aa(G, R, scene, grid, with_aa(cam, 1), W, H, S.default_lights(), p)
    c = render_aa(G, R, scene, grid, with_aa(cam, 0), W, H, S.default_lights(), p)
    assert all(np.array_equal(x, y) and np.array_equal(x, z) for x, y, z in zip(a, b, c))
    R.free(scene, grid)


def test_supersampled_equals_finer_raster_box_filter(G, R):
    # the device renders the finer raster and box-filters it: ids and AO
    # counts equal the plain render of the finer raster, colours its mean
    sc = S.globule(800, 760, 16.0, seed=5)
    W, H, m = 60, 45, 3
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=8, seed=1)
    scene, grid = R.upload(sc, lam=2.0)
    a_rgb, a_ids, a_vis = render_aa(G, R, scene, grid, with_aa(cam, m), W, H, S.default_lights(), p)
    f_rgb, f_ids, f_vis = render_aa(G, R, scene, grid, cam, m * W, m * H, S.default_lights(), p)
    assert np.array_equal(a_ids.ravel(), f_ids.ravel())
    assert np.array_equal(a_vis.ravel(), f_vis.ravel())
    box = f_rgb.reshape(H, m, W, m, 3).mean(axis=(1, 3)).reshape(-1, 3)
    assert np.abs(a_rgb - box).max() <= 2e-6
    R.free(scene, grid)


def test_supersampled_bands_and_host_outputs(G, R):
    import torch
    sc = S.globule(500, 475, 14.0, seed=3)
    lights = S.default_lights()
    W, H, m = 90, 77, 2
    scene, grid = R.upload(sc, lam=2.0)
    for prec in (S.PRECISION_FP32, S.PRECISION_FP64):
        p = S.Params(ao_samples=7, seed=5, precision=prec)
        cam = with_aa(S.ortho_camera(sc, W, H, angle_deg=20.0), m)
        ref = R.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
        dt = torch.float64 if prec == S.PRECISION_FP64 else torch.float32
        o = (torch.full((H, W, 3), -1, dtype=dt, device="cuda"),
             torch.full((m * H, m * W), -7, dtype=torch.int32, device="cuda"),
             torch.full((m * H, m * W), -7, dtype=torch.int32, device="cuda"))
        bands = [(0, 5), (5, 6), (6, 40), (40, 77)]
        for graph in (0, G.BATCH_GRAPH, G.BATCH_GRAPH):
            for t in o[1:]:
                t.fill_(-7)
            items = [G.make_item(scene, grid, cam, W, H, 7, lights, p, *o, rows=b) for b in bands[::-1]]
            G.gbrt_render_batch(R.ctx, items, graph)
            G.gbrt_sync(R.ctx)
            for x, y in zip(ref, o):
                assert torch.equal(x, y)
        host_rgb = np.zeros((H, W, 3), np.float64 if prec == S.PRECISION_FP64 else np.float32)
        host_ids = np.zeros((m * H, m * W), np.uint32)
        G.gbrt_render(R.ctx, scene, grid, cam, W, H, 7, lights, G.make_params(p, out_flags=G.HOST_PTRS),
                      host_rgb, host_ids)
        assert np.array_equal(host_rgb, ref[0].cpu().numpy())
        assert np.array_equal(host_ids, ref[1].cpu().numpy().view(np.uint32))
    R.free(scene, grid)


def test_supersampling_limits_rejected(G, R):
    import torch
    sc = S.globule(50, 40, 6.0, seed=1)
    scene, grid = R.upload(sc)
    W, H = 16, 16
    out = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    cam = S.ortho_camera(sc, W, H)
    p = G.make_params(S.Params(ao_samples=2))
    li = G.make_lights(S.default_lights())
    for bad in (-1, G.MAX_AA + 1):
        c = G.make_camera(cam)
        c.aa = bad
        with pytest.raises(G.GbrtError):
            G.gbrt_render(R.ctx, scene, grid, c, W, H, 2, li, p, out)
    # (m W)(m H) must stay below 2^31
    c = G.make_camera(cam)
    c.aa = 4
    with pytest.raises(G.GbrtError):
        G.gbrt_render(R.ctx, scene, grid, c, 65536, 2048, 2, li, p, out)
    R.free(scene, grid)
