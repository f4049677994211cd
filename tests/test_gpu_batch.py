"""Batched rendering: many frames of uneven size through one persistent launch
sequence (optionally replayed from a CUDA graph) give exactly the solo images."""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


def _frames(sc, n):
    out = []
    rng = np.random.default_rng(4)
    sizes = [(64, 48), (33, 17), (128, 96), (1, 1), (97, 61), (40, 40), (200, 30)]
    for k in range(n):
        W, H = sizes[k % len(sizes)]
        spp = int(rng.integers(1, 20))
        prec = S.PRECISION_FP64 if k % 4 == 3 else S.PRECISION_FP32
        out.append(dict(W=W, H=H, spp=spp, cam=S.ortho_camera(sc, W, H, angle_deg=37.0 * k),
                        p=S.Params(ao_samples=spp, seed=k, frame=k, precision=prec)))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_solo(G, graph):
    import torch
    sc = S.globule(500, 475, 14.0, seed=2)
    lights = S.default_lights()
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc, lam=2.0)
        fr = _frames(sc, 9)
        solo = []
        for f in fr:
            rgb, ids, vis = r.render(scene, grid, f["cam"], f["W"], f["H"], lights, f["p"], ids=True, vis=True)
            solo.append((rgb.clone(), ids.clone(), vis.clone()))
        outs = []
        items = []
        for f in fr:
            dt = torch.float64 if f["p"].precision == S.PRECISION_FP64 else torch.float32
            o = (torch.full((f["H"], f["W"], 3), -1, dtype=dt, device="cuda"),
                 torch.full((f["H"], f["W"]), -7, dtype=torch.int32, device="cuda"),
                 torch.full((f["H"], f["W"]), -7, dtype=torch.int32, device="cuda"))
            outs.append(o)
            items.append(G.make_item(scene, grid, f["cam"], f["W"], f["H"], f["spp"], lights, f["p"], *o))
        flags = G.BATCH_GRAPH if graph else 0
        for rep in range(3 if graph else 1):
            for o in outs:
                o[0].fill_(-1)
                o[1].fill_(-7)
            G.gbrt_render_batch(r.ctx, items, flags)
            G.gbrt_sync(r.ctx)
            for (a, b) in zip(solo, outs):
                for x, y in zip(a, b):
                    assert torch.equal(x, y)


def test_batch_with_two_scenes(G):
    import torch
    s1 = S.globule(300, 285, 10.0, seed=1)
    s2 = S.globule(900, 855, 18.0, seed=2)
    lights = S.default_lights()
    with G.Renderer(0) as r:
        a = r.upload(s1, lam=1.0)
        b = r.upload(s2, lam=4.0)
        jobs = [(a, s1, 50, 40, 7), (b, s2, 64, 64, 12), (a, s1, 31, 77, 3), (b, s2, 128, 16, 16)]
        items, outs, solo = [], [], []
        for (sg, sc, W, H, spp) in jobs:
            cam = S.ortho_camera(sc, W, H, 10.0 * spp)
            p = S.Params(ao_samples=spp, seed=spp)
            solo.append(r.render(sg[0], sg[1], cam, W, H, lights, p, ids=True)[:2])
            o = torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), dtype=torch.int32, device="cuda")
            outs.append(o)
            items.append(G.make_item(sg[0], sg[1], cam, W, H, spp, lights, p, o[0], o[1]))
        G.gbrt_render_batch(r.ctx, items)
        G.gbrt_sync(r.ctx)
        for (x0, x1), (y0, y1) in zip(solo, outs):
            assert torch.equal(x0, y0) and torch.equal(x1, y1)


def test_bands_equal_whole_frame(G):
    import torch
    sc = S.globule(500, 475, 14.0, seed=3)
    lights = S.default_lights()
    W, H = 90, 77
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc, lam=2.0)
        for prec in (S.PRECISION_FP32, S.PRECISION_FP64):
            p = S.Params(ao_samples=7, seed=5, precision=prec)
            cam = S.ortho_camera(sc, W, H, angle_deg=20.0)
            ref = r.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
            dt = torch.float64 if prec == S.PRECISION_FP64 else torch.float32
            o = (torch.full((H, W, 3), -1, dtype=dt, device="cuda"),
                 torch.full((H, W), -7, dtype=torch.int32, device="cuda"),
                 torch.full((H, W), -7, dtype=torch.int32, device="cuda"))
            bands = [(0, 5), (5, 6), (6, 40), (40, 77)]
            items = [G.make_item(scene, grid, cam, W, H, 7, lights, p, *o, rows=b) for b in bands[::-1]]
            G.gbrt_render_batch(r.ctx, items)
            G.gbrt_sync(r.ctx)
            for x, y in zip(ref, o):
                assert torch.equal(x, y)


def test_orbit64_graph_batch_sampled_vs_oracle(G, oracle):
    # the 64-frame orbit of the 26,318-object scene (512x512, 965x1137 and 1920x1080
    # frames, 8-32 AO samples, seed = frame index) as one graph-replayed batch, the
    # launch bench.py times; sampled pixels of frames of every size against the oracle
    import torch
    from gpu_common import assert_parity, compare
    w = S.paper_1mp()
    frames = S.orbit_frames(w.scene, 64)
    with G.Renderer(0) as r:
        scene, grid = r.upload(w.scene, lam=8.0)
        items, outs = [], []
        for f in frames:
            p = S.Params(ao_samples=f["spp"], seed=f["seed"], frame=f["frame"])
            o = (torch.full((f["height"], f["width"], 3), -1.0, device="cuda"),
                 torch.full((f["height"], f["width"]), -7, dtype=torch.int32, device="cuda"),
                 torch.full((f["height"], f["width"]), -7, dtype=torch.int32, device="cuda"))
            outs.append(o)
            items.append(G.make_item(scene, grid, f["camera"], f["width"], f["height"], f["spp"], w.lights, p, *o))
        for _ in range(2):  # capture, then replay
            G.gbrt_render_batch(r.ctx, items, G.BATCH_GRAPH)
            G.gbrt_sync(r.ctx)
        picked = {}
        for k, f in enumerate(frames):
            picked.setdefault((f["width"], f["height"]), []).append(k)
        assert len(picked) == 3
        rng = np.random.default_rng(64)
        for size, ks in sorted(picked.items()):
            for k in (ks[0], ks[-1]):
                f = frames[k]
                W, H = f["width"], f["height"]
                p = S.Params(ao_samples=f["spp"], seed=f["seed"], frame=f["frame"])
                pix = np.sort(rng.choice(W * H, 1500, replace=False))
                ref = oracle.render(w.scene, f["camera"], W, H, w.lights, p, pixels=pix, mode="grid", lam=2.0)
                rgb = outs[k][0].cpu().numpy().reshape(-1, 3).astype(np.float64)
                ids = outs[k][1].cpu().numpy().view(np.uint32).ravel()
                vis = outs[k][2].cpu().numpy().view(np.uint32).ravel()
                st = compare(rgb, ids, vis, ref, pixels=pix)
                assert_parity(st, f"orbit frame {k} {W}x{H} spp {f['spp']}")
                assert st["vis_eq"] >= 0.995, (k, st)
        r.free(scene, grid)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_batches_equal_solo(G, seed):
    # random mixes: two scenes, both precisions, supersampling, shadows, row
    # bands and ragged sizes in one batch (graph-replayed or not) give exactly
    # the solo renders
    import dataclasses
    import torch
    rng = np.random.default_rng(500 + seed)
    scenes = [S.globule(400, 380, 13.0, seed=seed), S.globule(150, 90, 8.0, seed=seed + 7)]
    lights = S.default_lights()
    with G.Renderer(0) as r:
        handles = [r.upload(sc, lam=float(rng.choice([1.0, 2.0, 8.0]))) for sc in scenes]
        items, outs, solo = [], [], []
        for k in range(int(rng.integers(5, 11))):
            si = int(rng.integers(0, 2))
            sc, (scene, grid) = scenes[si], handles[si]
            W, H = int(rng.integers(1, 80)), int(rng.integers(1, 60))
            m = int(rng.choice([1, 1, 2]))
            cam = dataclasses.replace(S.ortho_camera(sc, W, H, angle_deg=float(rng.uniform(0, 360))), aa=m)
            prec = S.PRECISION_FP64 if rng.random() < 0.3 else S.PRECISION_FP32
            p = S.Params(ao_samples=int(rng.integers(0, 12)), seed=int(rng.integers(0, 1 << 30)), frame=k,
                         precision=prec, shadows=bool(rng.random() < 0.5))
            ref = r.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
            solo.append(tuple(x.clone() for x in ref))
            dt = torch.float64 if prec == S.PRECISION_FP64 else torch.float32
            o = (torch.full((H, W, 3), -1, dtype=dt, device="cuda"),
                 torch.full((m * H, m * W), -7, dtype=torch.int32, device="cuda"),
                 torch.full((m * H, m * W), -7, dtype=torch.int32, device="cuda"))
            outs.append(o)
            if H > 2 and rng.random() < 0.5:
                cut = int(rng.integers(1, H))
                items.append(G.make_item(scene, grid, cam, W, H, p.ao_samples, lights, p, *o, rows=(cut, H)))
                items.append(G.make_item(scene, grid, cam, W, H, p.ao_samples, lights, p, *o, rows=(0, cut)))
            else:
                items.append(G.make_item(scene, grid, cam, W, H, p.ao_samples, lights, p, *o))
        order = rng.permutation(len(items))
        flags = G.BATCH_GRAPH if seed % 2 else 0
        for _ in range(2 if flags else 1):
            G.gbrt_render_batch(r.ctx, [items[i] for i in order], flags)
            G.gbrt_sync(r.ctx)
        for k, (a, b) in enumerate(zip(solo, outs)):
            for x, y in zip(a, b):
                assert torch.equal(x, y), k
