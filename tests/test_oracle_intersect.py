"""Pins of the oracle's ray-sphere and ray-cylinder tests.

Closed forms from geometry (a ray at perpendicular offset h from the centre or
axis) and, for random rays, the first sign change of each implicit surface
function found by dense sampling plus bisection -- a root finder that shares
nothing with the quadratic formulas under test.
"""
import math

import numpy as np
import pytest


def test_sphere_closed_form(oracle):
    c, r = np.array([1.0, -2.0, 3.0]), 1.7
    for h in [0.0, 0.3, 1.0, 1.69]:
        for D in [5.0, 40.0, 250.0]:
            o = c + np.array([h, 0.0, D])
            t, disc = oracle.hit_sphere(o, [0, 0, -1], c, r)
            assert t == pytest.approx(D - math.sqrt(r * r - h * h), rel=1e-13, abs=1e-12)
            assert disc == pytest.approx((r * r - h * h) / (r * r), rel=1e-9, abs=1e-12)
    # just outside the silhouette: a miss
    t, disc = oracle.hit_sphere(c + [r * 1.000001, 0, 10], [0, 0, -1], c, r)
    assert t is None and disc < 0
    # pointing away: miss
    t, _ = oracle.hit_sphere(c + [0, 0, 10], [0, 0, 1], c, r)
    assert t is None
    # origin inside: the far wall at distance r from the centre
    t, _ = oracle.hit_sphere(c, [0, 1, 0], c, r)
    assert t == pytest.approx(r, rel=1e-14)
    # tmax excludes the hit
    t, _ = oracle.hit_sphere(c + [0, 0, 10], [0, 0, -1], c, r, tmax=10 - r - 1e-9)
    assert t is None


def test_cylinder_closed_form(oracle):
    p0, p1, r = np.array([0.0, 0.0, 0.0]), np.array([4.0, 0.0, 0.0]), 0.3
    for s in [0.1, 2.0, 3.9]:
        for h in [0.0, 0.2, 0.29]:
            for D in [3.0, 90.0]:
                o = np.array([s, h, D])
                t, _ = oracle.hit_cylinder(o, [0, 0, -1], p0, p1, r)
                assert t == pytest.approx(D - math.sqrt(r * r - h * h), rel=1e-13, abs=1e-12)
    # past the end planes
    assert oracle.hit_cylinder([-0.01, 0, 5], [0, 0, -1], p0, p1, r)[0] is None
    assert oracle.hit_cylinder([4.01, 0, 5], [0, 0, -1], p0, p1, r)[0] is None
    # parallel to the axis, outside and inside: an open tube is never crossed
    assert oracle.hit_cylinder([-5, 1.0, 0], [1, 0, 0], p0, p1, r)[0] is None
    assert oracle.hit_cylinder([-5, 0.1, 0], [1, 0, 0], p0, p1, r)[0] is None
    # from inside the tube: the far wall at distance r
    t, _ = oracle.hit_cylinder([2.0, 0, 0], [0, 0, 1], p0, p1, r)
    assert t == pytest.approx(r, rel=1e-14)
    # oblique ray entering through the open end hits the inside wall:
    # from (-1, 0, 0) toward (3, 0.3, 0): the wall y = 0.3 is met at x = 3, inside [0, 4]
    d = np.array([4.0, 0.3, 0.0])
    t, _ = oracle.hit_cylinder([-1, 0, 0], d / np.linalg.norm(d), p0, p1, r)
    assert t == pytest.approx(np.linalg.norm(d), rel=1e-12)


def _first_root(f, tmax, n=20000):
    ts = np.linspace(1e-9, tmax, n)
    v = np.array([f(t) for t in ts])
    idx = np.nonzero(np.sign(v[1:]) != np.sign(v[:-1]))[0]
    if len(idx) == 0:
        return None
    a, b = ts[idx[0]], ts[idx[0] + 1]
    fa = f(a)
    for _ in range(80):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def test_sphere_random_rays_vs_bisection(oracle):
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(150):
        c = rng.uniform(-3, 3, 3)
        r = rng.uniform(0.5, 2.0)
        o = rng.uniform(-8, 8, 3)
        target = c + rng.uniform(-1.2, 1.2, 3) * r
        d = target - o
        d /= np.linalg.norm(d)
        t, disc = oracle.hit_sphere(o, d, c, r)
        if abs(disc) < 1e-3:
            continue
        ref = _first_root(lambda s: float(np.sum((o + s * d - c) ** 2) - r * r), 30.0)
        if ref is None:
            assert t is None
        else:
            assert t == pytest.approx(ref, abs=1e-6)
            checked += 1
    assert checked > 50


def test_cylinder_random_rays_vs_bisection(oracle):
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(150):
        p0 = rng.uniform(-2, 2, 3)
        ax = rng.standard_normal(3)
        ax /= np.linalg.norm(ax)
        L = rng.uniform(1.0, 4.0)
        p1 = p0 + L * ax
        r = rng.uniform(0.2, 1.0)
        o = rng.uniform(-8, 8, 3)
        target = p0 + rng.uniform(-0.2, 1.2) * L * ax + rng.uniform(-1.5, 1.5, 3) * r
        d = target - o
        d /= np.linalg.norm(d)
        t, disc = oracle.hit_cylinder(o, d, p0, p1, r)
        if abs(disc) < 1e-3:
            continue

        # implicit wall restricted to the segment: inside test via distance to the axis line;
        # a sign change only counts where the crossing's axial coordinate is in [0, L]
        def g(s):
            p = o + s * d - p0
            a = p @ ax
            return float(p @ p - a * a - r * r)

        ref = None
        ts = np.linspace(1e-9, 30.0, 30001)
        v = np.array([g(s) for s in ts])
        for k in np.nonzero(np.sign(v[1:]) != np.sign(v[:-1]))[0]:
            a, b = ts[k], ts[k + 1]
            fa = g(a)
            for _ in range(80):
                m = 0.5 * (a + b)
                if (g(m) > 0) == (fa > 0):
                    a, fa = m, g(m)
                else:
                    b = m
            root = 0.5 * (a + b)
            s_ax = (o + root * d - p0) @ ax
            if -1e-9 <= s_ax <= L + 1e-9:
                ref = root
                break
        if ref is None:
            assert t is None
        else:
            assert t == pytest.approx(ref, abs=1e-6)
            checked += 1
    assert checked > 40
