"""Pins of the oracle's camera, hit refinement and shading.

A lone sphere under an orthographic camera: at pixel (i, j) the ray hits the
point (u, v, sqrt(r^2 - u^2 - v^2)) with the outward normal p / r, and a lone
convex sphere has V = 1. The expected colour is built from that analytic
normal; the centre pixel (n = view vector) has the closed form
albedo (k_ao + s k_d sum_l l_z) + s k_s sum_l l_z^p.
"""
import math

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

W = H = 51
HALF = 2.55  # pixel pitch 0.1, pixel 25 sits on the axis


def cam():
    return S.Camera(eye=(0.0, 0.0, 10.0), dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), right=(1.0, 0.0, 0.0),
                    half_w=HALF, half_h=HALF)


def test_centre_pixel_closed_form(oracle):
    r = 2.0
    sc = S.make_scene([[0, 0, 0, r]], palette=[[0.8, 0.7, 0.6]])
    lights = S.default_lights()
    p = S.Params(ao_samples=8, precision=S.PRECISION_FP64)
    q = 25 * W + 25
    out = oracle.render(sc, cam(), W, H, lights, p, pixels=[q], mode="brute")
    assert out["id"][0] == 0
    assert out["t"][0] == pytest.approx(10.0 - r, abs=1e-12)
    assert out["vis"][0] == 8
    lz = [1 / math.sqrt(1.02), 0.5 / math.sqrt(5.25)]
    diff = 0.3 * 0.65 * sum(lz)
    spec = 0.3 * 0.4 * sum(z ** 40 for z in lz)
    expect = [min(1.0, a * (0.6 + diff) + spec) for a in (0.8, 0.7, 0.6)]
    assert np.allclose(out["rgb"][0], expect, atol=1e-7)


def rotated_cam(deg):
    a = math.radians(deg)
    back = np.array([math.sin(a), 0.0, math.cos(a)])
    right = np.array([math.cos(a), 0.0, -math.sin(a)])
    return S.Camera(eye=tuple(10.0 * back), dir=tuple(-back), up=(0.0, 1.0, 0.0), right=tuple(right),
                    half_w=HALF, half_h=HALF)


@pytest.mark.parametrize("deg", [0.0, 35.0, 200.0])
def test_off_axis_pixels_analytic_normal(oracle, deg):
    # camera rotated about +y: the pixel's offset from the axis through the
    # sphere centre is u right + v up, the hit point adds z (-dir)
    r = 2.0
    sc = S.make_scene([[0, 0, 0, r]], palette=[[0.5, 0.9, 0.3]])
    lights = S.default_lights()
    p = S.Params(ao_samples=4, precision=S.PRECISION_FP64)
    c = rotated_cam(deg)
    right, up, view = np.array(c.right), np.array(c.up), -np.array(c.dir)
    pix = [(25, 25), (30, 20), (12, 33), (40, 25), (25, 8), (7, 24), (38, 38)]
    qs = [j * W + i for i, j in pix]
    out = oracle.render(sc, c, W, H, lights, p, pixels=qs, mode="grid", lam=2.0)
    for k, (i, j) in enumerate(pix):
        u = 0.1 * (i + 0.5) - HALF
        v = HALF - 0.1 * (j + 0.5)
        z = math.sqrt(r * r - u * u - v * v)
        n = (u * right + v * up + z * view) / r
        assert out["t"][k] == pytest.approx(10.0 - z, abs=1e-10)
        spec = 0.0
        diff = 0.0
        for L in lights.dirs:
            L = np.array(L)
            ndl = n @ L
            if ndl > 0:
                diff += 0.3 * 0.65 * ndl
                refl = 2 * ndl * n - L
                spec += 0.3 * 0.4 * max(0.0, refl @ view) ** 40
        col = np.clip(np.array([0.5, 0.9, 0.3]) * (0.6 + diff) + spec, 0, 1)
        assert np.allclose(out["rgb"][k], col, atol=1e-9), (i, j)


def test_rows_start_at_top_and_columns_at_left(oracle):
    sc = S.make_scene([[1.0, 1.0, 0.0, 0.8]])
    out = oracle.render(sc, cam(), W, H, S.default_lights(), S.Params(ao_samples=0), mode="brute")
    hit = (out["id"] != oracle.MISS).reshape(H, W)
    jj, ii = np.nonzero(hit)
    assert hit.sum() > 100
    assert ii.min() > 25 and jj.max() < 25


def test_background_and_clamp(oracle):
    sc = S.make_scene([[0, 0, 0, 2.0]], palette=[[1.0, 1.0, 1.0]])
    lights = S.default_lights()
    lights.skylight = 5.0
    p = S.Params(ao_samples=2, background=(0.1, 0.2, 0.3))
    out = oracle.render(sc, cam(), W, H, lights, p, pixels=[0, 25 * W + 25], mode="brute")
    assert out["id"][0] == oracle.MISS
    assert np.allclose(out["rgb"][0], [0.1, 0.2, 0.3])
    assert np.allclose(out["rgb"][1], [1.0, 1.0, 1.0])


def test_zero_samples_means_open_sky(oracle):
    sc = S.make_scene([[0, 0, 0, 2.0], [0, 0, 2.5, 0.4]])
    p0 = S.Params(ao_samples=0)
    out = oracle.render(sc, cam(), W, H, S.default_lights(), p0, pixels=[25 * W + 20], mode="brute")
    p1 = S.Params(ao_samples=4096)
    ref = oracle.render(sc, cam(), W, H, S.default_lights(), p1, pixels=[25 * W + 20], mode="brute")
    assert out["vis"][0] == 0
    assert np.all(out["rgb"][0] >= ref["rgb"][0] - 1e-12)


def test_direct_light_shadow_of_a_sphere(oracle):
    # sphere B sits between sphere A and light 1 (straight toward the camera
    # side): points of A whose ray toward light 1 meets B lose light 1; the
    # blocked set is found here by the closed-form line-sphere distance
    rA, rB = 2.0, 0.9
    L1 = np.array([0.0, 0.0, 1.0])
    L2 = np.array([0.6, 0.0, 0.8])
    lights = S.Lights(dirs=[tuple(L1), tuple(L2)], intensity=[1.0, 1.0])
    B = np.array([0.3, 0.2, 4.0])
    sc = S.make_scene([[0, 0, 0, rA], [B[0], B[1], B[2], rB]], palette=[[0.7, 0.6, 0.5]])
    c = rotated_cam(30.0)   # looks at A from the side so B does not hide A's centre
    right, up, view = np.array(c.right), np.array(c.up), -np.array(c.dir)
    pix, expect = [], []
    for i in range(5, 46, 4):
        for j in range(5, 46, 4):
            u, v = 0.1 * (i + 0.5) - HALF, HALF - 0.1 * (j + 0.5)
            if u * u + v * v >= (0.97 * rA) ** 2:
                continue
            z = math.sqrt(rA * rA - u * u - v * v)
            n = (u * right + v * up + z * view) / rA
            pnt = rA * n
            # the camera ray must meet A first (B is elsewhere along it)
            o = pnt + 10.0 * view
            f = o - B
            b = f @ (-view)
            if (f @ f - b * b) < rB * rB and b < 0:
                continue
            diff = spec = 0.0
            for Ld in (L1, L2):
                ndl = n @ Ld
                if ndl <= 0:
                    continue
                fb = pnt + 1e-3 * n - B
                bb = fb @ Ld
                blocked = (fb @ fb - bb * bb) < rB * rB and bb < 0
                if blocked:
                    continue
                diff += 0.3 * 0.65 * ndl
                refl = 2 * ndl * n - Ld
                spec += 0.3 * 0.4 * max(0.0, refl @ view) ** 40
            pix.append(j * W + i)
            expect.append(np.clip(np.array([0.7, 0.6, 0.5]) * (0.6 + diff) + spec, 0, 1))
    p = S.Params(ao_samples=0, shadows=True, precision=S.PRECISION_FP64)
    out = oracle.render(sc, c, W, H, lights, p, pixels=pix, mode="brute")
    assert np.all(out["id"] == 0)
    assert np.allclose(out["rgb"], np.array(expect), atol=1e-9)
    # some of the sampled points are in B's shadow, some are not
    p0 = S.Params(ao_samples=0, shadows=False, precision=S.PRECISION_FP64)
    unshadowed = oracle.render(sc, c, W, H, lights, p0, pixels=pix, mode="brute")
    changed = np.any(np.abs(unshadowed["rgb"] - out["rgb"]) > 1e-6, axis=1)
    assert 0 < changed.sum() < len(pix)
