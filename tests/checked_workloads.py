"""Workloads rendered through the checked build of the library.

Run by tests/test_gpu_checked.py in a process of its own with
GBRT_LIB_VARIANT=checked: libgbrt_checked.so tests every index that comes
from data (cells, items, object ids, hit slots, pixels) against its buffer,
and gbrt_sync raises GBRT_EBOUNDS if any fell outside. Each workload below is
followed by a sync, so the first one that strays names itself. The small
globule is also compared with the oracle: the checks change no result.
Prints one line per workload and "checked ok" at the end.
"""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_0801_1500_gb300 import gbrt as G  # noqa: E402
from paper_0801_1500_gb300 import scenes as S  # noqa: E402

assert G.LIB_PATH.endswith("libgbrt_checked.so"), G.LIB_PATH

FP32, FP64 = S.PRECISION_FP32, S.PRECISION_FP64


def step(r, name):
    G.gbrt_sync(r.ctx)   # raises GbrtError(GBRT_EBOUNDS) on a stray index
    print("ok", name, flush=True)


def main():
    import oracle
    from gpu_common import assert_parity, compare, gpu_frame
    lights = S.default_lights()
    small = S.small_fp64()
    paper = S.paper_scene(0)
    with G.Renderer(0) as r:
        # the small globule in both precisions, against the oracle
        sc, gr = r.upload(small.scene, lam=2.0)
        for prec in (FP32, FP64):
            p = S.Params(ao_samples=8, seed=0, precision=prec)
            got = gpu_frame(G, r, sc, gr, small.camera, 256, 256, lights, p)
            ref = oracle.render(small.scene, small.camera, 256, 256, lights, p, mode="brute")
            assert_parity(compare(*got, ref), f"checked build, small globule, precision {prec}")
            step(r, f"small globule precision {prec} (parity with the oracle)")
        # ragged frames, the largest width and height, 4,096 samples with shadows
        for W, H, spp, shadows in ((1, 1, 5, False), (97, 61, 9, False), (65536, 1, 2, False), (1, 65536, 2, False),
                                   (24, 20, 4096, True)):
            cam = S.ortho_camera(small.scene, W, H, angle_deg=30.0)
            r.render(sc, gr, cam, W, H, lights, S.Params(ao_samples=spp, seed=1, shadows=shadows), ids=True,
                     vis=True)
            step(r, f"{W}x{H} {spp} spp shadows={shadows}")
        # supersampled pinhole views
        for prec in (FP32, FP64):
            cam = S.pinhole_camera(small.scene, 80, 60, angle_deg=40.0, aa=3)
            r.render(sc, gr, cam, 80, 60, lights, S.Params(ao_samples=4, seed=2, precision=prec), ids=True, vis=True)
            step(r, f"pinhole 3x3 supersampled precision {prec}")
        # the AO probe
        pts = torch.from_numpy(np.array([[0.0, 0.0, 30.0], [5.0, 5.0, 26.0]])).cuda()
        nrm = torch.from_numpy(np.array([[0.0, 0.0, 1.0], [0.0, 0.6, 0.8]])).cuda()
        out = torch.empty(2, dtype=torch.float32, device="cuda")
        for prec in (FP32, FP64):
            G.gbrt_ao_probe(r.ctx, sc, gr, pts, nrm, 4096, S.Params(seed=3, precision=prec), out)
            step(r, f"AO probe precision {prec}")
        # the allocation-free render
        stream = torch.cuda.current_stream()
        for prec in (FP32, FP64):
            dt = torch.float64 if prec == FP64 else torch.float32
            outs = (torch.empty((120, 200, 3), dtype=dt, device="cuda"),
                    torch.empty((120, 200), dtype=torch.int32, device="cuda"),
                    torch.empty((120, 200), dtype=torch.int32, device="cuda"))
            cam = S.ortho_camera(small.scene, 200, 120, angle_deg=15.0)
            G.gbrt_render_noalloc(sc, gr, cam, 200, 120, 6, lights, S.Params(ao_samples=6, seed=4, precision=prec),
                                  *outs, stream=stream)
            torch.cuda.synchronize()
            step(r, f"allocation-free render precision {prec}")

        # the paper-sized scene: both precisions, shadows
        ps, pg = r.upload(paper, lam=8.0)
        cam = S.ortho_camera(paper, 965, 1137)
        for prec, shadows in ((FP32, False), (FP64, False), (FP32, True)):
            r.render(ps, pg, cam, 965, 1137, lights, S.Params(ao_samples=16, seed=0, precision=prec, shadows=shadows),
                     ids=True, vis=True)
            step(r, f"paper-sized precision {prec} shadows={shadows}")
        # a batch of uneven frames of two scenes (the AO walk's per-ray scene
        # pointers), with a band, replayed through a graph
        items, keep = [], []
        for k, (h, scn, W, H, spp) in enumerate(((pg, paper, 512, 512, 12), (gr, small.scene, 200, 150, 7),
                                                  (pg, paper, 320, 700, 20))):
            handle_s, handle_g = (ps, pg) if h is pg else (sc, gr)
            o = (torch.empty((H, W, 3), device="cuda"), torch.empty((H, W), dtype=torch.int32, device="cuda"))
            keep.append(o)
            rows = (H // 4, H // 2) if k == 2 else None
            items.append(G.make_item(handle_s, handle_g, S.ortho_camera(scn, W, H, 20.0 * k), W, H, spp, lights,
                                     S.Params(ao_samples=spp, seed=k), o[0], o[1], rows=rows))
        for graph in (0, G.BATCH_GRAPH, G.BATCH_GRAPH):
            G.gbrt_render_batch(r.ctx, items, graph)
            step(r, f"two-scene batch (graph={bool(graph)})")
        r.free(ps, pg)

        # an animated scene: device-side update and rebuild, then render
        base = S.globule(800, 760, 16.0, seed=5)
        traj = S.MDTrajectory(base, amplitude=0.3, spin_deg=5.0, seed=2)
        ms, mg = r.upload(base, lam=2.0)
        for k in range(1, 4):
            fr = traj.frame(k)
            G.gbrt_scene_update(r.ctx, ms, torch.from_numpy(fr.spheres).cuda(), torch.from_numpy(fr.cylinders).cuda())
            G.gbrt_grid_rebuild(r.ctx, mg, ms)
            r.render(ms, mg, S.ortho_camera(base, 90, 70), 90, 70, lights, S.Params(ao_samples=5, seed=k), ids=True)
            step(r, f"animation frame {k}")
        r.free(ms, mg)

        # the largest serving scene (250k objects)
        big = S.serving_scenes(8, 1000, 250000, seed=0)[7]
        bs, bg = r.upload(big, lam=8.0)
        r.render(bs, bg, S.ortho_camera(big, 640, 480, angle_deg=30.0), 640, 480, lights,
                 S.Params(ao_samples=16, seed=3), ids=True, vis=True)
        step(r, "250k-object scene")
        r.free(bs, bg)
        r.free(sc, gr)
    print("checked ok", flush=True)


if __name__ == "__main__":
    main()
