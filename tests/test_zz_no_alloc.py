"""The allocation-free render entry point gives the same frames as gbrt_render.

gbrt_render_noalloc is for callers that cannot allocate device memory while
they render (an application whose own allocator holds the free device memory,
or a loop that must not call cudaMalloc/cudaFree). It keeps its working data in
a fixed array inside the library, so two calls in a row must not leak state
into each other. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S
from gpu_common import assert_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


def _flat(rgb, ids, vis):
    return (rgb.cpu().numpy().reshape(-1, 3).astype(np.float64), ids.cpu().numpy().view(np.uint32).ravel(),
            vis.cpu().numpy().view(np.uint32).ravel())


def test_noalloc_matches_render_on_two_calls_in_a_row(G):
    import torch
    sc = S.globule(2000, 1900, 25.0, seed=0)
    lights = S.default_lights()
    frames = [(256, 256, S.Params(ao_samples=8, seed=0, precision=S.PRECISION_FP32), 0.0),
              (200, 120, S.Params(ao_samples=5, seed=3, frame=2, precision=S.PRECISION_FP64), 40.0)]
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc, lam=2.0)
        stream = torch.cuda.current_stream()
        outs = []
        for W, H, p, ang in frames:
            cam = S.ortho_camera(sc, W, H, angle_deg=ang)
            ref = r.render(scene, grid, cam, W, H, lights, p, ids=True, vis=True)
            G.gbrt_sync(r.ctx)
            dt = torch.float64 if p.precision == S.PRECISION_FP64 else torch.float32
            got = (torch.full((H, W, 3), -1.0, dtype=dt, device="cuda"),
                   torch.full((H, W), -7, dtype=torch.int32, device="cuda"),
                   torch.full((H, W), -7, dtype=torch.int32, device="cuda"))
            G.gbrt_render_noalloc(scene, grid, cam, W, H, p.ao_samples, lights, p, *got, stream=stream)
            outs.append((ref, got))
        torch.cuda.synchronize()
        for ref, got in outs:
            a, b = _flat(*ref), _flat(*got)
            # same kernels, same inputs: identical; and within the parity tolerance
            assert all(np.array_equal(x, y) for x, y in zip(a, b))
            st = compare(b[0], b[1], b[2], {"rgb": a[0], "id": a[1], "vis": a[2],
                                           "grazing": np.zeros(len(a[1]), bool)})
            assert st["id_mismatch"] == 0 and st["frac_bad"] == 0.0 and st["mae"] <= 1e-4, st


def test_noalloc_rejects_frames_above_its_limit(G):
    import torch
    sc = S.make_scene([[0, 0, 0, 1.0]])
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc)
        W, H = 512, 256
        assert W * H > G.NOALLOC_MAX_PIXELS
        out = torch.empty((H, W, 3), device="cuda")
        with pytest.raises(G.GbrtError) as e:
            G.gbrt_render_noalloc(scene, grid, S.ortho_camera(sc, W, H), W, H, 4, S.default_lights(),
                                  S.Params(), out)
        assert e.value.code == G.EINVAL


def test_noalloc_rejects_supersampling(G):
    import dataclasses

    import torch
    sc = S.make_scene([[0, 0, 0, 1.0]])
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc)
        W, H = 32, 32
        out = torch.empty((H, W, 3), device="cuda")
        cam = dataclasses.replace(S.ortho_camera(sc, W, H), aa=2)
        with pytest.raises(G.GbrtError) as e:
            G.gbrt_render_noalloc(scene, grid, cam, W, H, 4, S.default_lights(), S.Params(), out)
        assert e.value.code == G.EINVAL


def test_noalloc_allocates_nothing_and_matches_the_oracle(G, oracle):
    # after one call of each precision (the set-up, and the first launch of
    # each kernel), twenty calls of mixed size and precision change neither
    # torch's allocations nor the device's free memory; one of the frames is
    # checked against the FP64 oracle directly
    import torch
    sc = S.globule(600, 570, 15.0, seed=7)
    lights = S.default_lights()
    sizes = [(256, 256), (97, 61), (1, 1), (200, 120), (17, 301)]
    precs = [S.PRECISION_FP32, S.PRECISION_FP64]
    with G.Renderer(0) as r:
        scene, grid = r.upload(sc, lam=2.0)
        stream = torch.cuda.current_stream()
        outs = {}
        for W, H in sizes:
            for prec in precs:
                dt = torch.float64 if prec == S.PRECISION_FP64 else torch.float32
                outs[W, H, prec] = (torch.empty((H, W, 3), dtype=dt, device="cuda"),
                                    torch.empty((H, W), dtype=torch.int32, device="cuda"),
                                    torch.empty((H, W), dtype=torch.int32, device="cuda"))

        def call(k, W, H, prec):
            p = S.Params(ao_samples=3 + k % 6, seed=k, frame=k, precision=prec, shadows=bool(k % 3 == 0))
            cam = S.ortho_camera(sc, W, H, angle_deg=13.0 * k)
            G.gbrt_render_noalloc(scene, grid, cam, W, H, p.ao_samples, lights, p, *outs[W, H, prec], stream=stream)
            return cam, p

        for k, prec in enumerate(precs):
            call(3 * k, *sizes[0], prec)   # shadows on: every kernel of the path runs once per precision
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        last = None
        for k in range(20):
            W, H = sizes[k % len(sizes)]
            prec = precs[(k // len(sizes)) % 2]
            last = (W, H, prec) + call(k, W, H, prec)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        W, H, prec, cam, p = last
        rgb, ids, vis = outs[W, H, prec]
        ref = oracle.render(sc, cam, W, H, lights, p, mode="brute")
        st = compare(rgb.cpu().numpy().reshape(-1, 3).astype(np.float64), ids.cpu().numpy().view(np.uint32).ravel(),
                     vis.cpu().numpy().view(np.uint32).ravel(), ref)
        assert_parity(st, "noalloc vs oracle")
        r.free(scene, grid)


def test_noalloc_after_update_and_rebuild_ordered_by_an_event(G):
    # the scene and grid change on the context's stream; the caller's stream
    # waits on an event recorded there, then renders without allocating: the
    # same frame as gbrt_render on the context
    import torch
    base = S.globule(800, 760, 16.0, seed=5)
    traj = S.MDTrajectory(base, amplitude=0.3, spin_deg=5.0, seed=2)
    W, H = 90, 70
    lights = S.default_lights()
    p = S.Params(ao_samples=5, seed=1)
    ctx_stream = torch.cuda.Stream()
    caller = torch.cuda.Stream()
    with G.Renderer(0, ctx_stream) as r:
        scene, grid = r.upload(base, lam=2.0)
        cam = S.ortho_camera(base, W, H)
        for k in range(1, 4):
            fr = traj.frame(k)
            G.gbrt_scene_update(r.ctx, scene, fr.spheres, fr.cylinders)
            G.gbrt_grid_rebuild(r.ctx, grid, scene)
            ev = torch.cuda.Event()
            ev.record(ctx_stream)
            caller.wait_event(ev)
            got = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), dtype=torch.int32, device="cuda"))
            G.gbrt_render_noalloc(scene, grid, cam, W, H, 5, lights, p, *got, stream=caller)
            caller.synchronize()
            ref = r.render(scene, grid, cam, W, H, lights, p, ids=True)
            G.gbrt_sync(r.ctx)
            assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1]), k
        r.free(scene, grid)
