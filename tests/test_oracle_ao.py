"""Pins of the oracle's ambient occlusion.

* A lone convex object sees an unoccluded sky: every AO sample escapes.
* A point on a plane next to a sphere of radius R resting on that plane, at
  horizontal distance d from the contact point, sees the sphere with the
  point-to-sphere form factor F = cos(theta) R^2 / D^2 (sphere fully above the
  horizon), D^2 = d^2 + R^2, cos(theta) = R / D, so the unoccluded cosine-
  weighted fraction is V = 1 - R^3 / (d^2 + R^2)^(3/2).
* A point facing a fully visible sphere of radius R_B at distance D, at angle
  theta from the normal: V = 1 - cos(theta) R_B^2 / D^2.
Monte-Carlo bound: |V_hat - V| <= 4 sqrt(V (1 - V) / N).
"""
import math

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

N = 65536


@pytest.mark.parametrize("mode", ["brute", "grid"])
def test_sphere_on_plane(oracle, mode):
    R = 2.0
    sc = S.make_scene([[0.0, 0.0, R, R]])
    dists = np.array([0.5, 1.0, 2.0, 4.0, 8.0]) * R
    pts = np.stack([dists, np.zeros_like(dists), np.zeros_like(dists)], 1)
    nrm = np.tile([0.0, 0.0, 1.0], (len(dists), 1))
    v = oracle.ao_probe(sc, pts, nrm, N, seed=3, mode=mode, eps=1e-6)
    expect = 1.0 - R ** 3 / (dists ** 2 + R ** 2) ** 1.5
    bound = 4 * np.sqrt(expect * (1 - expect) / N)
    assert np.all(np.abs(v - expect) <= bound), (v, expect, bound)


def test_point_facing_sphere(oracle):
    # sphere A at the origin (radius 1), probe points on A; sphere B fully visible
    RA, RB = 1.0, 0.8
    B = np.array([0.0, 0.0, 5.0])
    sc = S.make_scene([[0, 0, 0, RA], [B[0], B[1], B[2], RB]])
    cases = []
    for ang in [0.0, 20.0, 45.0, 60.0]:
        a = math.radians(ang)
        n = np.array([math.sin(a), 0.0, math.cos(a)])
        p = RA * n
        to_b = B - p
        D = np.linalg.norm(to_b)
        cos_t = (to_b @ n) / D
        # B must lie fully above the tangent plane at p
        assert (to_b @ n) > RB
        cases.append((p, n, 1 - cos_t * RB ** 2 / D ** 2))
    pts = np.array([c[0] for c in cases])
    nrm = np.array([c[1] for c in cases])
    v = oracle.ao_probe(sc, pts, nrm, N, seed=11, mode="grid", lam=4.0, eps=1e-6)
    expect = np.array([c[2] for c in cases])
    bound = 4 * np.sqrt(expect * (1 - expect) / N)
    assert np.all(np.abs(v - expect) <= bound), (v, expect)


def test_lone_objects_see_open_sky(oracle):
    lights = S.default_lights()
    # the tube's axis is perpendicular to the view, so no ray enters an open end
    # and every hit is on the outer wall (an open tube seen end-on is not convex)
    for sc in [S.make_scene([[0.0, 0.0, 0.0, 2.0]]),
               S.make_scene(None, [[-3, -1, 0, 3, 1, 0.0, 0.7]])]:
        cam = S.ortho_camera(sc, 48, 40)
        p = S.Params(ao_samples=16, precision=S.PRECISION_FP64)
        for mode in ("brute", "grid"):
            out = oracle.render(sc, cam, 48, 40, lights, p, mode=mode)
            hit = out["id"] != oracle.MISS
            assert hit.sum() > 200
            assert np.all(out["vis"][hit] == 16)


def test_probe_matches_render_sampling(oracle):
    # AO of a rendered pixel equals the probe at its refined point: same counter (pixel, s, frame)
    sc = S.globule(300, 285, 10.0, seed=4)
    W, H = 40, 30
    cam = S.ortho_camera(sc, W, H)
    p = S.Params(ao_samples=32, seed=77, frame=5)
    out = oracle.render(sc, cam, W, H, S.default_lights(), p, mode="grid")
    # a pixel whose hit is a sphere seen head-on: rebuild its hit point from t
    q = int(np.nonzero((out["id"] < 300) & ~out["grazing"])[0][len(out["id"]) // 7 % 50])
    i, j = q % W, q // W
    u = cam.half_w * (2 * (i + 0.5) / W - 1)
    v = cam.half_h * (1 - 2 * (j + 0.5) / H)
    o = np.array(cam.eye) + u * np.array(cam.right) + v * np.array(cam.up)
    d = np.array(cam.dir)
    ph = o + out["t"][q] * d
    c = sc.spheres[out["id"][q], :3].astype(np.float64)
    n = (ph - c) / np.linalg.norm(ph - c)
    ph = c + sc.spheres[out["id"][q], 3] * n
    # the probe indexes its points 0..n-1; pad so that our point sits at index q
    pts = np.zeros((q + 1, 3))
    nrm = np.tile([0.0, 0.0, 1.0], (q + 1, 1))
    pts[q], nrm[q] = ph, n
    vis = oracle.ao_probe(sc, pts, nrm, 32, seed=77, frame=5, mode="grid")
    assert vis[q] * 32 == pytest.approx(out["vis"][q], abs=1e-9)
