"""GPU parity tests: the CUDA path through the C ABI against the FP64 oracle."""
import dataclasses
import math

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


def test_philox_matches_oracle_and_known_answers(G, R, oracle):
    import torch
    rng = np.random.default_rng(0)
    n = 4099
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0], key[0] = 0, 0
    ctr[1], key[1] = 0xFFFFFFFF, 0xFFFFFFFF
    ctr[2] = [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]
    key[2] = [0xa4093822, 0x299f31d0]
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    G.gbrt_philox4x32_10(R.ctx, dc, dk, out)
    G.gbrt_sync(R.ctx)
    got = out.cpu().numpy().view(np.uint32)
    for k in range(0, n, 37):
        assert list(got[k]) == list(oracle.philox4x32_10(ctr[k], key[k]))
    assert list(got[0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert list(got[2]) == [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0, 4.0])
def test_grid_matches_oracle_grid(G, R, oracle, lam):
    sc = S.globule(2000, 1900, 25.0, seed=0)
    scene, grid = R.upload(sc, lam=lam)
    gi = G.gbrt_grid_info(grid)
    oi = oracle.grid_info(sc, lam)
    assert gi["dims"] == oi["dims"]
    # the device lists an object only in cells its shape reaches (a subset of
    # the cells its box overlaps, which is what the oracle's grid uses)
    assert 0.4 * oi["refs"] <= gi["refs"] <= oi["refs"]
    assert np.allclose(gi["lo"], oi["lo"], atol=1e-4) and np.allclose(gi["hi"], oi["hi"], atol=1e-4)
    R.free(scene, grid)


@pytest.mark.parametrize("prec", [S.PRECISION_FP64, S.PRECISION_FP32])
def test_small_globule_full_frame(G, R, oracle, prec):
    # 2,000 spheres + 1,900 cylinders, 256x256, 8 AO samples (plain FP64 and FP32 paths)
    w = S.small_fp64()
    p = S.Params(ao_samples=8, seed=0, precision=prec)
    scene, grid = R.upload(w.scene, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p)
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, p, mode="brute")
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, "small")
    if prec == S.PRECISION_FP64:
        assert st["vis_eq"] >= 0.9999
    R.free(scene, grid)


@pytest.mark.parametrize("shift", [(300.0, -200.0, 500.0), (-2000.0, 1500.0, 800.0)])
@pytest.mark.parametrize("prec", [S.PRECISION_FP64, S.PRECISION_FP32])
def test_scene_far_from_the_origin(G, R, oracle, prec, shift):
    # the small globule moved hundreds to thousands of units off the origin
    # (molecular coordinates are often hundreds of angstroms): the float
    # scene records and the FP32 walk lose absolute precision there, the
    # parity rule must still hold against the oracle's brute force
    w = S.small_fp64()
    off = np.array(shift, np.float32)
    sp = w.scene.spheres.copy()
    sp[:, :3] += off
    cy = w.scene.cylinders.copy()
    cy[:, :3] += off
    cy[:, 3:6] += off
    sc = dataclasses.replace(w.scene, spheres=sp, cylinders=cy)
    cam = S.ortho_camera(sc, w.width, w.height, angle_deg=25.0)
    p = S.Params(ao_samples=8, seed=0, precision=prec)
    scene, grid = R.upload(sc, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, w.width, w.height, w.lights, p)
    ref = oracle.render(sc, cam, w.width, w.height, w.lights, p, mode="brute")
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, f"globule moved by {shift}")
    R.free(scene, grid)


@pytest.mark.parametrize("W,H,spp", [(97, 61, 9), (33, 131, 3), (1, 1, 5), (17, 1, 4)])
@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_ragged_frames(G, R, oracle, W, H, spp, prec):
    sc = S.globule(600, 570, 15.0, seed=7)
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=spp, seed=11, frame=3, precision=prec)
    scene, grid = R.upload(sc, lam=1.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="brute")
    assert_parity(compare(rgb, ids, vis, ref), f"{W}x{H} spp {spp}")
    R.free(scene, grid)


@pytest.mark.parametrize("spp,shadows", [(1, False), (255, False), (1000, False), (4096, True)])
def test_sample_counts_up_to_the_bound(G, R, oracle, spp, shadows):
    # up to GBRT_MAX_SAMPLES AO samples a pixel (with shadows, a hit's job list
    # is its samples plus one ray per light it faces): every job maps back to
    # its hit and sample, so the AO counts equal the oracle's
    w = S.small_fp64()
    W, H = 24, 20
    cam = S.ortho_camera(w.scene, W, H, angle_deg=10.0)
    p = S.Params(ao_samples=spp, seed=5, precision=S.PRECISION_FP32, shadows=shadows)
    scene, grid = R.upload(w.scene, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, w.lights, p)
    ref = oracle.render(w.scene, cam, W, H, w.lights, p, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, f"{spp} samples")
    hit = ref["id"] != oracle.MISS
    assert int(vis.max()) <= spp and int(vis[hit].max()) > 0
    assert st["vis_eq"] >= 0.99
    R.free(scene, grid)


@pytest.mark.parametrize("W,H", [(65536, 1), (1, 65536)])
def test_largest_width_and_height(G, R, oracle, W, H):
    # the largest accepted width / height: one line of pixels across the scene
    sc = S.globule(600, 570, 15.0, seed=7)
    # square pixels, the line spanning the globule
    half = 16.0
    cam = S.Camera(eye=(0.0, 0.0, 40.0), dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), right=(1.0, 0.0, 0.0),
                   half_w=half * min(1.0, W / H), half_h=half * min(1.0, H / W))
    p = S.Params(ao_samples=2, seed=5)
    scene, grid = R.upload(sc, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="grid", lam=2.0)
    assert 0.5 < (ref["id"] != 0xFFFFFFFF).mean() < 1.0
    assert_parity(compare(rgb, ids, vis, ref), f"{W}x{H}")
    R.free(scene, grid)


@pytest.fixture(scope="module")
def paper(G, R):
    w = S.paper_1mp()
    scene, grid = R.upload(w.scene, lam=8.0)  # the density bench.py's autotuner picks
    yield w, scene, grid
    R.free(scene, grid)


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_paper_scene_1mp_full_frame(G, R, oracle, paper, prec):
    # 26,318 objects, 965x1137, 16 AO samples: every pixel against the oracle's grid walk
    w, scene, grid = paper
    p = S.Params(ao_samples=16, seed=0, precision=prec)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p)
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, p, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref)
    print("paper 1.1MP", "fp64" if prec else "fp32", st)
    assert_parity(st, "paper 1mp")


def test_paper_scene_1mp_sampled_vs_brute_force(G, R, oracle, paper):
    # sampled pixels against the brute-force definition (no grid on the oracle
    # side); 4,000 pixels, so the 99.9% rule allows 4 beyond 1/255
    w, scene, grid = paper
    p = S.Params(ao_samples=16, seed=0, precision=S.PRECISION_FP32)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p)
    pix = np.random.default_rng(1).choice(w.width * w.height, 4000, replace=False)
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, p, pixels=pix, mode="brute")
    assert_parity(compare(rgb, ids, vis, ref, pixels=pix), "paper 1mp vs brute force")


def test_paper_scene_17mp_centre_crop(G, R, oracle, paper):
    # 3860x4548, 16 AO samples; per-pixel error map on the 256x256 centre crop
    w, scene, grid = paper
    w2 = S.paper_17mp(scene=w.scene)
    p = S.Params(ao_samples=16, seed=0, precision=S.PRECISION_FP32)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w2.camera, w2.width, w2.height, w2.lights, p)
    j0, i0 = w2.height // 2 - 128, w2.width // 2 - 128
    jj, ii = np.meshgrid(np.arange(j0, j0 + 256), np.arange(i0, i0 + 256), indexing="ij")
    pix = (jj * w2.width + ii).ravel()
    ref = oracle.render(w2.scene, w2.camera, w2.width, w2.height, w2.lights, p, pixels=pix, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref, pixels=pix)
    print("17.6MP crop", st)
    assert_parity(st, "17mp crop")
    # sampled pixels over the whole frame
    pix = np.random.default_rng(2).choice(w2.width * w2.height, 4000, replace=False)
    ref = oracle.render(w2.scene, w2.camera, w2.width, w2.height, w2.lights, p, pixels=pix, mode="grid", lam=2.0)
    assert_parity(compare(rgb, ids, vis, ref, pixels=pix), "17mp sampled")


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_ao_probe_sphere_on_plane(G, R, oracle, prec):
    import torch
    Rr = 2.0
    sc = S.make_scene([[0.0, 0.0, Rr, Rr]])
    scene, grid = R.upload(sc, lam=1.0)
    dists = np.array([0.5, 1.0, 2.0, 4.0, 8.0]) * Rr
    pts = np.stack([dists, 0 * dists, 0 * dists], 1)
    nrm = np.tile([0.0, 0.0, 1.0], (len(dists), 1))
    N = 65536
    p = S.Params(seed=3, precision=prec, eps=1e-6)
    out = torch.empty(len(dists), dtype=torch.float32, device="cuda")
    G.gbrt_ao_probe(R.ctx, scene, grid, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), N, p, out)
    G.gbrt_sync(R.ctx)
    v = out.cpu().numpy().astype(np.float64)
    expect = 1.0 - Rr ** 3 / (dists ** 2 + Rr ** 2) ** 1.5
    assert np.all(np.abs(v - expect) <= 4 * np.sqrt(expect * (1 - expect) / N)), (v, expect)
    ref = oracle.ao_probe(sc, pts, nrm, N, seed=3, eps=1e-6, mode="brute")
    assert np.all(np.abs(v - ref) * N <= 2), (v, ref)  # same samples: at most a couple of flips
    R.free(scene, grid)


def test_lone_sphere_sees_open_sky(G, R):
    sc = S.make_scene([[0.0, 0.0, 0.0, 2.0]])
    cam = S.ortho_camera(sc, 80, 60)
    scene, grid = R.upload(sc)
    for prec in (S.PRECISION_FP32, S.PRECISION_FP64):
        _, ids, vis = gpu_frame(G, R, scene, grid, cam, 80, 60, S.default_lights(),
                                S.Params(ao_samples=32, precision=prec))
        hit = ids != G.MISS
        assert hit.sum() > 1000 and np.all(vis[hit] == 32)
    R.free(scene, grid)


def test_empty_scene_renders_background(G, R):
    sc = S.make_scene(np.zeros((0, 4)))
    scene, grid = R.upload(sc)
    cam = S.Camera(eye=(0, 0, 5), dir=(0, 0, -1), up=(0, 1, 0), right=(1, 0, 0), half_w=1, half_h=1)
    p = S.Params(ao_samples=4, background=(0.25, 0.5, 0.75))
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, 40, 30, S.default_lights(), p)
    assert np.all(ids == G.MISS) and np.allclose(rgb, [0.25, 0.5, 0.75])
    R.free(scene, grid)


def test_invalid_arguments_rejected(G, R):
    import torch
    bad = S.make_scene([[0, 0, 0, float("nan")]])
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_scene_upload(R.ctx, bad.spheres, bad.cylinders, bad.color_idx, bad.palette)
    assert e.value.code == G.EINVAL
    # the device-pointer path validates in its prep kernel
    d = torch.tensor([[0.0, 0.0, 0.0, -1.0]], device="cuda")
    with pytest.raises(G.GbrtError):
        G.gbrt_scene_upload(R.ctx, d, torch.zeros((0, 7), device="cuda"),
                            torch.zeros(1, dtype=torch.int32, device="cuda"), torch.ones((1, 3), device="cuda"),
                            G.DEVICE_PTRS)
    zero_len = S.make_scene(None, [[1, 1, 1, 1, 1, 1, 0.3]])
    with pytest.raises(G.GbrtError):
        G.gbrt_scene_upload(R.ctx, zero_len.spheres, zero_len.cylinders, zero_len.color_idx, zero_len.palette)
    sc = S.make_scene([[0, 0, 0, 1.0]])
    scene, grid = R.upload(sc)
    cam = S.ortho_camera(sc, 8, 8)
    out = torch.empty((8, 8, 3), device="cuda")
    for W, H, spp in [(0, 8, 4), (8, -1, 4), (8, 8, -1), (8, 8, 100000), (65537, 1, 4), (1, 65537, 4),
                      (65536, 32768, 4)]:   # width, height <= 65536 and width * height < 2^31
        with pytest.raises(G.GbrtError) as e:
            G.gbrt_render(R.ctx, scene, grid, cam, W, H, spp, S.default_lights(), S.Params(), out)
        assert e.value.code == G.EINVAL
    # a grid built for another scene (another object count) would list ids
    # past this scene's arrays: rejected by render, batch and probe
    other = S.globule(40, 35, 5.0, seed=3)
    o_scene, o_grid = R.upload(other)
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_render(R.ctx, scene, o_grid, cam, 8, 8, 4, S.default_lights(), S.Params(), out)
    assert e.value.code == G.EINVAL
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_render_batch(R.ctx, [G.make_item(o_scene, grid, cam, 8, 8, 4, S.default_lights(), S.Params(), out)])
    assert e.value.code == G.EINVAL
    pts = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    vis = torch.empty(1, device="cuda")
    with pytest.raises(G.GbrtError) as e:
        G.gbrt_ao_probe(R.ctx, o_scene, grid, pts, pts, 4, S.Params(), vis)
    assert e.value.code == G.EINVAL
    G.gbrt_sync(R.ctx)
    R.free(o_scene, o_grid)
    R.free(scene, grid)


def test_host_output_pointers(G, R):
    import torch
    sc = S.globule(300, 285, 10.0, seed=9)
    W, H = 70, 50
    cam = S.ortho_camera(sc, W, H)
    scene, grid = R.upload(sc)
    p = S.Params(ao_samples=6, seed=2)
    dev_rgb, dev_ids, _ = R.render(scene, grid, cam, W, H, S.default_lights(), p, ids=True)
    G.gbrt_sync(R.ctx)
    host_rgb = np.zeros((H, W, 3), np.float32)
    host_ids = np.zeros((H, W), np.uint32)
    G.gbrt_render(R.ctx, scene, grid, cam, W, H, 6, S.default_lights(), G.make_params(p, out_flags=G.HOST_PTRS),
                  host_rgb, host_ids)
    assert np.array_equal(host_rgb, dev_rgb.cpu().numpy())
    assert np.array_equal(host_ids, dev_ids.cpu().numpy().view(np.uint32))
    R.free(scene, grid)


def test_asynchronous_host_outputs(G, R):
    # three frames enqueued back to back into page-locked host buffers, one
    # wait at the end: each equals its synchronous render
    import torch
    sc = S.globule(300, 285, 10.0, seed=9)
    W, H = 70, 50
    cam = S.ortho_camera(sc, W, H)
    scene, grid = R.upload(sc)
    frames = [S.Params(ao_samples=6, seed=s, frame=s) for s in (1, 2, 3)]
    outs = [(torch.empty((H, W, 3), dtype=torch.float32).pin_memory().numpy(),
             torch.empty((H, W), dtype=torch.int32).pin_memory().numpy().view(np.uint32)) for _ in frames]
    for p, (rgb, ids) in zip(frames, outs):
        G.gbrt_render(R.ctx, scene, grid, cam, W, H, 6, S.default_lights(),
                      G.make_params(p, out_flags=G.HOST_PTRS | G.HOST_ASYNC), rgb, ids)
    G.gbrt_sync(R.ctx)
    for p, (rgb, ids) in zip(frames, outs):
        ref_rgb, ref_ids = np.zeros((H, W, 3), np.float32), np.zeros((H, W), np.uint32)
        G.gbrt_render(R.ctx, scene, grid, cam, W, H, 6, S.default_lights(), G.make_params(p, out_flags=G.HOST_PTRS),
                      ref_rgb, ref_ids)
        assert np.array_equal(rgb, ref_rgb) and np.array_equal(ids, ref_ids)
    assert not np.array_equal(outs[0][0], outs[1][0])  # different seeds, different AO
    # a longer stream of frames of changing sizes (the two staging buffers
    # alternate and grow mid-stream) with all three outputs, against renders
    # into device memory
    sizes = [(70, 50), (90, 64), (70, 50), (128, 80), (33, 17), (128, 80), (90, 64)]
    outs = []
    for k, (w, h) in enumerate(sizes):
        p = S.Params(ao_samples=5, seed=10 + k, frame=k)
        o = (torch.empty((h, w, 3), dtype=torch.float32).pin_memory().numpy(),
             torch.empty((h, w), dtype=torch.int32).pin_memory().numpy().view(np.uint32),
             torch.empty((h, w), dtype=torch.int32).pin_memory().numpy().view(np.uint32))
        outs.append(o)
        G.gbrt_render(R.ctx, scene, grid, S.ortho_camera(sc, w, h, angle_deg=15.0 * k), w, h, 5,
                      S.default_lights(), G.make_params(p, out_flags=G.HOST_PTRS | G.HOST_ASYNC), *o)
    G.gbrt_sync(R.ctx)
    for k, ((w, h), o) in enumerate(zip(sizes, outs)):
        p = S.Params(ao_samples=5, seed=10 + k, frame=k)
        ref = R.render(scene, grid, S.ortho_camera(sc, w, h, angle_deg=15.0 * k), w, h, S.default_lights(), p,
                       ids=True, vis=True)
        G.gbrt_sync(R.ctx)
        assert np.array_equal(o[0], ref[0].cpu().numpy()), k
        assert np.array_equal(o[1], ref[1].cpu().numpy().view(np.uint32)), k
        assert np.array_equal(o[2], ref[2].cpu().numpy().view(np.uint32)), k
    # a change of the context's stream between asynchronous renders: the
    # copies of the earlier ones still complete before the next gbrt_sync
    side = torch.cuda.Stream()
    outs2 = []
    for k, strm in enumerate((None, side, None)):
        if strm is not None:
            G.gbrt_set_stream(R.ctx, strm)
        p = S.Params(ao_samples=5, seed=30 + k, frame=k)
        o = torch.empty((50, 70, 3), dtype=torch.float32).pin_memory().numpy()
        outs2.append((p, o))
        G.gbrt_render(R.ctx, scene, grid, cam, W, H, 5, S.default_lights(),
                      G.make_params(p, out_flags=G.HOST_PTRS | G.HOST_ASYNC), o)
    G.gbrt_set_stream(R.ctx, R.stream)
    G.gbrt_sync(R.ctx)
    for p, o in outs2:
        ref = R.render(scene, grid, cam, W, H, S.default_lights(), p)[0]
        G.gbrt_sync(R.ctx)
        assert np.array_equal(o, ref.cpu().numpy())
    with pytest.raises(G.GbrtError):  # asynchronous outputs must be host outputs
        G.gbrt_render(R.ctx, scene, grid, cam, W, H, 6, S.default_lights(),
                      G.make_params(frames[0], out_flags=G.HOST_ASYNC), torch.empty((H, W, 3), device="cuda"))
    R.free(scene, grid)


def test_deterministic_and_grid_invariant(G, R, oracle):
    # the same frame twice is bit-identical; across grid densities the hit ids
    # are identical on every non-grazing pixel (the result must not depend on
    # the grid) and each frame meets the parity rule
    sc = S.globule(800, 760, 16.0, seed=5)
    W, H = 120, 90
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=8, seed=1)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="brute")
    ok = ~ref["grazing"]
    frames = []
    for lam in (0.25, 0.5, 1.0, 2.0, 8.0):
        scene, grid = R.upload(sc, lam=lam)
        a = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
        b = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        assert_parity(compare(*a, ref), f"lambda {lam}")
        frames.append(a)
        R.free(scene, grid)
    for f in frames[1:]:
        assert np.array_equal(f[1][ok], frames[0][1][ok])


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_open_tube_inner_wall(G, R, oracle, prec):
    # seen obliquely, an open tube shows its inner wall through the end, whose AO
    # rays meet the opposite wall of the same tube
    sc = S.make_scene(None, [[-3, -1, 0, 3, 1, 0.5, 0.7]])
    W, H = 64, 40
    cam = S.ortho_camera(sc, W, H, angle_deg=70.0)
    p = S.Params(ao_samples=16, seed=4, precision=prec)
    scene, grid = R.upload(sc)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="brute")
    hit = ref["id"] != oracle.MISS
    assert (ref["vis"][hit] < 16).sum() > 20  # the case under test occurs
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, "open tube")
    assert st["vis_eq"] >= 0.995, st
    R.free(scene, grid)


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_pinhole_camera_inside_an_atom(G, R, oracle, prec):
    sc = S.globule(400, 380, 12.0, seed=6)
    c = sc.spheres[17, :3].astype(np.float64)
    cam = S.Camera(eye=tuple(c), dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), right=(1.0, 0.0, 0.0),
                   half_w=0.8, half_h=0.6, kind=S.CAMERA_PINHOLE)
    W, H = 48, 36
    p = S.Params(ao_samples=8, seed=9, precision=prec)
    scene, grid = R.upload(sc, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="brute")
    assert_parity(compare(rgb, ids, vis, ref), "pinhole inside an atom")
    R.free(scene, grid)


@pytest.mark.parametrize("prec", [S.PRECISION_FP32, S.PRECISION_FP64])
def test_direct_light_shadows_small(G, R, oracle, prec):
    w = S.small_fp64()
    p = S.Params(ao_samples=8, seed=0, precision=prec, shadows=True)
    scene, grid = R.upload(w.scene, lam=2.0)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p)
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, p, mode="brute")
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, "shadows small")
    # shadows change the image
    p0 = S.Params(ao_samples=8, seed=0, precision=prec, shadows=False)
    rgb0, _, _ = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p0)
    assert (np.abs(rgb0 - rgb).max(axis=1) > 1e-3).mean() > 0.05
    R.free(scene, grid)


def test_direct_light_shadows_paper_scene(G, R, oracle, paper):
    w, scene, grid = paper
    p = S.Params(ao_samples=16, seed=0, precision=S.PRECISION_FP32, shadows=True)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, w.camera, w.width, w.height, w.lights, p)
    ref = oracle.render(w.scene, w.camera, w.width, w.height, w.lights, p, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref)
    print("paper 1.1MP shadows", st)
    assert_parity(st, "shadows paper")


@pytest.mark.parametrize("lam", [2.0, 8.0])
def test_largest_serving_scene(G, R, oracle, lam):
    # the 250k-object scene of the serving trace (the largest grid: up to
    # 2M cells at lambda 8), pinhole view from outside, FP32 path vs the oracle
    sc = S.globule(127500, 121125, 60.0 * (127500 / 13500.0) ** (1.0 / 3.0), seed=1)
    W, H = 192, 160
    cam = S.pinhole_camera(sc, W, H, angle_deg=25.0, fov_deg=35.0)
    p = S.Params(ao_samples=4, seed=7)
    scene, grid = R.upload(sc, lam=lam)
    rgb, ids, vis = gpu_frame(G, R, scene, grid, cam, W, H, S.default_lights(), p)
    ref = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="grid", lam=2.0)
    st = compare(rgb, ids, vis, ref)
    assert_parity(st, f"250k objects lambda {lam}")
    assert st["vis_eq"] >= 0.999
    assert 0.3 < (ref["id"] != 0xFFFFFFFF).mean() < 0.95
    R.free(scene, grid)


def test_phase_times_in_both_profiling_modes(G, R):
    # all kernels timed: the primary, AO walk and shading times are positive
    # and the AO plan (inside the primary kernel) is 0; AO-walk mode: only the
    # AO walk is timed, close to its time in the full mode
    import torch
    sc = S.globule(2000, 1900, 25.0, seed=0)
    W, H = 256, 256
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=8, seed=0)
    scene, grid = R.upload(sc, lam=8.0)
    out = torch.empty((H, W, 3), device="cuda")
    args = (R.ctx, scene, grid, G.make_camera(cam), W, H, 8, G.make_lights(S.default_lights()), G.make_params(p), out)
    with pytest.raises(G.GbrtError):
        fresh = G.Renderer(0)
        try:
            G.gbrt_phase_times(fresh.ctx)   # nothing timed yet
        finally:
            fresh.close()
    times = {}
    for mode in ("all", "ao_walk"):
        G.gbrt_set_profiling(R.ctx, True, ao_walk_only=mode == "ao_walk")
        runs = []
        for _ in range(5):
            G.gbrt_render(*args)
            runs.append(G.gbrt_phase_times(R.ctx))
        G.gbrt_set_profiling(R.ctx, False)
        times[mode] = runs[-1]
    a, w = times["all"], times["ao_walk"]
    assert a["primary"] > 0 and a["ao_walk"] > 0 and a["shade"] > 0 and a["ao_plan"] >= 0
    assert w["primary"] == -1 and w["ao_plan"] == -1 and w["shade"] == -1 and w["ao_walk"] > 0
    assert 0.5 * a["ao_walk"] < w["ao_walk"] < 2.0 * a["ao_walk"]
    G.gbrt_sync(R.ctx)
    R.free(scene, grid)
