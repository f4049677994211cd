"""Pins of the oracle's supersampling (m x m regular sub-pixel grid, box filter).

1. A lone sphere seen by an orthographic and by a pinhole camera: every
   sub-sample's hit or miss, its distance and its colour follow from the
   sphere equation and the analytic normal (a lone convex sphere has V = 1), so
   the pixel colour is the mean of m^2 closed-form values, background where the
   sub-sample misses. Pixels straddling the silhouette test the sub-pixel
   positions (a + 0.5)/m and the averaging.
2. A supersampled render equals the box filter of the plain render of the
   m-times finer raster: the same rays (up to the rounding of the sub-pixel
   position), the same Philox counters (the finer raster's pixel index), so the
   same hit ids and AO counts, and colours whose mean is the pixel colour.
"""
import math

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

W = H = 51
HALF = 2.55   # pixel pitch 0.1
R = 2.0
ALBEDO = np.array([0.5, 0.9, 0.3])
BG = (0.1, 0.2, 0.3)


def _colour(n, view, lights):
    diff = spec = 0.0
    for L in lights.dirs:
        L = np.array(L)
        ndl = n @ L
        if ndl > 0:
            diff += 0.3 * 0.65 * ndl
            refl = 2 * ndl * n - L
            spec += 0.3 * 0.4 * max(0.0, refl @ view) ** 40
    return np.clip(ALBEDO * (0.6 + diff) + spec, 0, 1)


def _half(kind):
    # orthographic: half extents in scene units; pinhole: tangents of the half angles
    return HALF if kind == S.CAMERA_ORTHO else HALF / 10.0


def _cam(kind, m):
    return S.Camera(eye=(0.0, 0.0, 10.0), dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), right=(1.0, 0.0, 0.0),
                    half_w=_half(kind), half_h=_half(kind), kind=kind, aa=m)


def _expected(kind, m, i, j, lights):
    """Closed-form sub-samples of pixel (i, j), sub-row major: (hit, t, rgb, disc)."""
    eye = np.array([0.0, 0.0, 10.0])
    hw = _half(kind)
    subs = []
    for b in range(m):
        for a in range(m):
            u = hw * (2.0 * (i + (a + 0.5) / m) / W - 1.0)
            v = hw * (1.0 - 2.0 * (j + (b + 0.5) / m) / H)
            if kind == S.CAMERA_ORTHO:
                o, d = eye + np.array([u, v, 0.0]), np.array([0.0, 0.0, -1.0])
            else:
                o, d = eye, np.array([u, v, -1.0]) / math.sqrt(u * u + v * v + 1.0)
            # |o + t d|^2 = R^2 with |d| = 1: t = -(o.d) - sqrt((o.d)^2 - (|o|^2 - R^2))
            bq = o @ d
            disc = bq * bq - (o @ o - R * R)
            if disc <= 0:
                subs.append((False, math.inf, np.array(BG), disc))
                continue
            t = -bq - math.sqrt(disc)
            n = (o + t * d) / R
            subs.append((True, t, _colour(n, -d, lights), disc))
    return subs


@pytest.mark.parametrize("kind", [S.CAMERA_ORTHO, S.CAMERA_PINHOLE])
@pytest.mark.parametrize("m", [2, 3, 4])
def test_sphere_silhouette_closed_form(oracle, kind, m):
    sc = S.make_scene([[0, 0, 0, R]], palette=[ALBEDO.tolist()])
    lights = S.default_lights()
    p = S.Params(ao_samples=4, precision=S.PRECISION_FP64, background=BG)
    pix, exp = [], []
    for j in range(0, H, 2):
        for i in range(0, W, 3):
            e = _expected(kind, m, i, j, lights)
            # skip pixels with a sub-sample within rounding of the silhouette
            if any(abs(s[3]) < 1e-6 for s in e):
                continue
            pix.append((i, j))
            exp.append(e)
    partial = sum(1 for e in exp if 0 < sum(s[0] for s in e) < m * m)
    assert partial >= 6, "pick pixels across the silhouette"
    qs = [j * W + i for i, j in pix]
    out = oracle.render(sc, _cam(kind, m), W, H, lights, p, pixels=qs, mode="brute")
    assert out["id"].shape == (len(qs) * m * m,)
    for k, e in enumerate(exp):
        for s, (hit, t, rgb, _) in enumerate(e):
            idx = k * m * m + s
            assert (out["id"][idx] == 0) == hit, (pix[k], s)
            if hit:
                assert out["t"][idx] == pytest.approx(t, abs=1e-10)
                assert out["vis"][idx] == 4
        mean = np.mean([s[2] for s in e], axis=0)
        assert np.allclose(out["rgb"][k], mean, atol=1e-9), pix[k]
    assert out["counters"]["primary_rays"] == len(qs) * m * m


@pytest.mark.parametrize("m", [2, 3])
@pytest.mark.parametrize("shadows", [False, True])
def test_supersampled_equals_box_filter_of_finer_raster(oracle, m, shadows):
    sc = S.globule(60, 50, 8.0, seed=3)
    w0, h0 = 14, 11
    lights = S.default_lights()
    p = S.Params(ao_samples=8, precision=S.PRECISION_FP64, seed=77, frame=5, shadows=shadows)
    cam = S.ortho_camera(sc, w0, h0, angle_deg=30.0)
    cam_aa = S.Camera(**{**cam.__dict__, "aa": m})
    fine = oracle.render(sc, cam, w0 * m, h0 * m, lights, p, mode="grid", lam=2.0)
    ss = oracle.render(sc, cam_aa, w0, h0, lights, p, mode="grid", lam=2.0)
    fw = w0 * m
    for j in range(h0):
        for i in range(w0):
            k = j * w0 + i
            cols = []
            for b in range(m):
                for a in range(m):
                    qf = (m * j + b) * fw + (m * i + a)
                    s = k * m * m + b * m + a
                    if not fine["grazing"][qf]:
                        assert ss["id"][s] == fine["id"][qf], (i, j, a, b)
                        assert ss["vis"][s] == fine["vis"][qf], (i, j, a, b)
                    cols.append(fine["rgb"][qf])
            if not any(fine["grazing"][(m * j + b) * fw + m * i + a] for b in range(m) for a in range(m)):
                assert np.allclose(ss["rgb"][k], np.mean(cols, axis=0), atol=1e-9), (i, j)
    hits = int((ss["id"] != 0xFFFFFFFF).sum())
    assert 0 < hits < ss["id"].size
    assert ss["counters"]["ao_rays"] == fine["counters"]["ao_rays"]
