"""GPU tests of the animation path: gbrt_scene_update + gbrt_grid_rebuild
(device-side grid rebuild per molecular-dynamics frame) against fresh
uploads and host builds of the same frames, and against the FP64 oracle."""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import assert_parity, compare, gpu_frame

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


def fresh(G, R, sc, lam, cam, W, H, lights, p):
    scene, grid = R.upload(sc, lam=lam)
    out = gpu_frame(G, R, scene, grid, cam, W, H, lights, p)
    info = G.gbrt_grid_info(grid)
    R.free(scene, grid)
    return out, info


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_rebuilt_grid_equals_host_build(G, R, prec):
    base = S.globule(2000, 1900, 25.0, seed=0)
    traj = S.MDTrajectory(base, amplitude=0.4, spin_deg=7.0, seed=1)
    W, H = 128, 96
    lights = S.default_lights()
    p = S.Params(ao_samples=6, seed=3, precision=prec)
    scene, grid = R.upload(base, lam=2.0)
    for k in range(1, 6):
        fr = traj.frame(k)
        cam = S.ortho_camera(fr, W, H)
        G.gbrt_scene_update(R.ctx, scene, fr.spheres, fr.cylinders)
        G.gbrt_grid_rebuild(R.ctx, grid, scene)
        got = gpu_frame(G, R, scene, grid, cam, W, H, lights, p)
        ref, info = fresh(G, R, fr, 2.0, cam, W, H, lights, p)
        gi = G.gbrt_grid_info(grid)
        # the device computes the same geometry and lists as a host build
        assert gi["dims"] == info["dims"] and gi["refs"] == info["refs"], (k, gi, info)
        assert np.allclose(gi["lo"], info["lo"]) and np.allclose(gi["hi"], info["hi"])
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), k
    R.free(scene, grid)


def test_device_array_update_and_graph_replay(G, R):
    import torch
    base = S.globule(800, 760, 16.0, seed=5)
    traj = S.MDTrajectory(base, amplitude=0.3, spin_deg=5.0, seed=2)
    W, H = 90, 70
    lights = S.default_lights()
    p = S.Params(ao_samples=5, seed=1)
    scene, grid = R.upload(base, lam=2.0)
    out = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), dtype=torch.int32, device="cuda"),
           torch.empty((H, W), dtype=torch.int32, device="cuda"))
    for k in range(1, 5):
        fr = traj.frame(k)
        cam = S.ortho_camera(base, W, H)   # fixed camera: the molecule turns in view
        G.gbrt_scene_update(R.ctx, scene, torch.from_numpy(fr.spheres).cuda(), torch.from_numpy(fr.cylinders).cuda())
        G.gbrt_grid_rebuild(R.ctx, grid, scene)
        # one captured graph, replayed for every frame: the grid patch pass
        # picks up each rebuild's geometry
        G.gbrt_render_batch(R.ctx, [G.make_item(scene, grid, cam, W, H, 5, lights, p, *out)], G.BATCH_GRAPH)
        G.gbrt_sync(R.ctx)
        got = (out[0].cpu().numpy().reshape(-1, 3).astype(np.float64), out[1].cpu().numpy().view(np.uint32).ravel(),
               out[2].cpu().numpy().view(np.uint32).ravel())
        ref, _ = fresh(G, R, fr, 2.0, cam, W, H, lights, p)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), k
    R.free(scene, grid)


def test_rebuild_overflow_is_reported_then_recovers(G, R):
    base = S.globule(600, 570, 14.0, seed=4)
    W, H = 64, 48
    lights = S.default_lights()
    p = S.Params(ao_samples=4, seed=0)
    scene, grid = R.upload(base, lam=2.0)
    G.gbrt_grid_rebuild(R.ctx, grid, scene)   # allocates with 1.5x headroom
    G.gbrt_sync(R.ctx)
    fat = S.Scene(spheres=base.spheres.copy(), cylinders=base.cylinders.copy(), color_idx=base.color_idx,
                  palette=base.palette)
    fat.spheres[:, 3] *= 4.0                  # each atom now reaches many more cells
    G.gbrt_scene_update(R.ctx, scene, fat.spheres, fat.cylinders)
    G.gbrt_grid_rebuild(R.ctx, grid, scene)
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_sync(R.ctx)
    assert e.value.code == G.ECAPACITY
    G.gbrt_grid_rebuild(R.ctx, grid, scene)   # sees the overflow, grows, rebuilds
    G.gbrt_sync(R.ctx)
    cam = S.ortho_camera(fat, W, H)
    got = gpu_frame(G, R, scene, grid, cam, W, H, lights, p)
    ref, info = fresh(G, R, fat, 2.0, cam, W, H, lights, p)
    assert G.gbrt_grid_info(grid)["refs"] == info["refs"]
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    R.free(scene, grid)


def test_update_rejects_bad_geometry(G, R):
    import torch
    base = S.globule(100, 90, 8.0, seed=6)
    scene, grid = R.upload(base, lam=2.0)
    bad = base.spheres.copy()
    bad[3, 3] = -1.0
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_scene_update(R.ctx, scene, bad, base.cylinders)
    assert e.value.code == G.EINVAL
    bad = base.spheres.copy()
    bad[5, 0] = np.nan
    G.gbrt_scene_update(R.ctx, scene, torch.from_numpy(bad).cuda(), torch.from_numpy(base.cylinders).cuda())
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_sync(R.ctx)
    assert e.value.code == G.EINVAL
    # a good update afterwards restores the scene
    G.gbrt_scene_update(R.ctx, scene, base.spheres, base.cylinders)
    G.gbrt_grid_rebuild(R.ctx, grid, scene)
    G.gbrt_sync(R.ctx)
    other = S.globule(50, 40, 6.0, seed=1)
    o_scene, o_grid = R.upload(other)
    with pytest.raises(G.GbrtError):
        G.gbrt_grid_rebuild(R.ctx, grid, o_scene)   # another object count
    R.free(o_scene, o_grid)
    R.free(scene, grid)


def test_paper_scene_md_frame_vs_oracle(G, R, oracle):
    # 26,318 objects, 12 device-side updates + rebuilds, then the FP32 path vs the oracle
    base = S.paper_scene()
    traj = S.MDTrajectory(base, amplitude=0.3, seed=0)
    W, H = 965, 1137
    lights = S.default_lights()
    p = S.Params(ao_samples=16, seed=0, frame=12)
    scene, grid = R.upload(base, lam=8.0)
    for k in range(1, 13):
        fr = traj.frame(k)
        G.gbrt_scene_update(R.ctx, scene, fr.spheres, fr.cylinders)
        G.gbrt_grid_rebuild(R.ctx, grid, scene)
    cam = S.ortho_camera(fr, W, H)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, lights, p)
    rng = np.random.default_rng(5)
    pixels = np.sort(rng.choice(W * H, 4000, replace=False))
    ref = oracle.render(fr, cam, W, H, lights, p, pixels=pixels, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref, pixels)
    assert_parity(st, "md frame 12")
    assert st["vis_eq"] >= 0.999
    R.free(scene, grid)
