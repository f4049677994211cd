"""Pins of the oracle's uniform grid and 3D-DDA.

The nearest hit is defined over all objects; the grid walk must give the same
object and distance for every grid density. The cells a ray visits must cover
every cell its path passes through (checked by dense sampling of the path) and
consecutive cells must be face neighbours.
"""
import math

import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S


def tiny_scene(seed, n_sph=60, n_cyl=40, box=6.0):
    rng = np.random.default_rng(seed)
    sph = np.concatenate([rng.uniform(-box, box, (n_sph, 3)), rng.uniform(0.3, 1.5, (n_sph, 1))], 1)
    p0 = rng.uniform(-box, box, (n_cyl, 3))
    ax = rng.standard_normal((n_cyl, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    p1 = p0 + ax * rng.uniform(0.5, 4.0, (n_cyl, 1))
    cyl = np.concatenate([p0, p1, rng.uniform(0.1, 0.6, (n_cyl, 1))], 1)
    return S.make_scene(sph, cyl)


def random_rays(seed, n, box=6.0):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-2 * box, 2 * box, (n, 3))
    tgt = rng.uniform(-box, box, (n, 3))
    d = tgt - o
    # a few axis-parallel rays (zero direction components)
    d[: n // 10, 1] = 0.0
    d[: n // 20, 0] = 0.0
    return o, d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("lam", [0.25, 1.0, 8.0])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid_equals_brute_force(oracle, lam, seed):
    sc = tiny_scene(seed)
    o, d = random_rays(100 + seed, 3000)
    ib, tb, gb, _ = oracle.nearest(sc, o, d, mode="brute")
    ig, tg, gg, _ = oracle.nearest(sc, o, d, mode="grid", lam=lam)
    assert (ib != oracle.MISS).sum() > 500
    ok = ~gb
    assert np.array_equal(ib[ok], ig[ok])
    hit = ok & (ib != oracle.MISS)
    assert np.array_equal(tb[hit], tg[hit])


def test_ray_starting_inside_grid(oracle):
    sc = tiny_scene(7)
    rng = np.random.default_rng(8)
    o = rng.uniform(-4, 4, (2000, 3))
    d = rng.standard_normal((2000, 3))
    ib, tb, gb, _ = oracle.nearest(sc, o, d, mode="brute")
    ig, tg, gg, _ = oracle.nearest(sc, o, d, mode="grid", lam=2.0)
    assert np.array_equal(ib[~gb], ig[~gb])


def test_tie_break_lower_id(oracle):
    # two identical spheres and a sphere/cylinder pair touching the ray at the same t
    sc = S.make_scene([[0, 0, 0, 1.0], [0, 0, 0, 1.0]])
    ids, ts, _, _ = oracle.nearest(sc, [[0, 0, 5]], [[0, 0, -1]], mode="brute")
    assert ids[0] == 0 and ts[0] == pytest.approx(4.0)
    ids2, _, _, _ = oracle.nearest(sc, [[0, 0, 5]], [[0, 0, -1]], mode="grid", lam=4.0)
    assert ids2[0] == 0
    # cylinder ids follow sphere ids
    sc = S.make_scene([[5, 5, 5, 0.5]], [[-1, 0, 0, 1, 0, 0, 0.5]])
    ids, _, _, _ = oracle.nearest(sc, [[0, 0, 5]], [[0, 0, -1]], mode="brute")
    assert ids[0] == 1


def _cells_on_path(info, o, d, t0, t1, n=200000):
    lo, hi = info["lo"], info["hi"]
    dims = np.array(info["dims"])
    h = (hi - lo) / dims
    ts = np.linspace(t0, t1, n)
    p = o[None, :] + ts[:, None] * d[None, :]
    inside = np.all((p > lo + 1e-9) & (p < hi - 1e-9), axis=1)
    c = np.floor((p[inside] - lo) / h).astype(np.int64)
    # skip samples within 1e-7 of a cell boundary (either side is a valid answer there)
    frac = (p[inside] - lo) / h - c
    clean = np.all((frac > 1e-7) & (frac < 1 - 1e-7), axis=1)
    c = c[clean]
    c = np.clip(c, 0, dims - 1)
    return set(((c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]).tolist())


@pytest.mark.parametrize("lam", [0.5, 4.0])
def test_dda_visits_every_cell_on_the_path(oracle, lam):
    sc = tiny_scene(3)
    info = oracle.grid_info(sc, lam)
    rng = np.random.default_rng(11)
    dims = np.array(info["dims"])
    for k in range(40):
        o = rng.uniform(-15, 15, 3)
        d = rng.uniform(-8, 8, 3) - o
        if k % 7 == 0:
            d[k % 3] = 0.0
        d /= np.linalg.norm(d)
        cells, _ = oracle.grid_walk(sc, o, d, lam=lam)
        visited = set(cells.tolist())
        expect = _cells_on_path(info, o, d, 0.0, 60.0)
        assert expect <= visited
        assert len(visited) == len(cells)  # no cell visited twice
        # consecutive cells share a face
        zyx = np.stack([cells // (dims[0] * dims[1]), (cells // dims[0]) % dims[1], cells % dims[0]], 1)
        if len(cells) > 1:
            steps = np.abs(np.diff(zyx, axis=0)).sum(1)
            assert np.all(steps == 1)


@pytest.mark.parametrize("lam", [125.0, 1000.0, 8000.0])
@pytest.mark.parametrize("yz", [(4.0, 0.3), (3.0, -3.0)])
def test_walk_counts_cells_up_to_the_hit_cell(oracle, lam, yz):
    # One sphere (radius 5 at the origin) listed in every cell of its box; a
    # ray along +x at offset (y, z) meets it at x = -sqrt(25 - y^2 - z^2). The
    # nearest-hit walk must count every cell from the box face to the cell
    # holding that point -- earlier cells list the sphere too, and testing it
    # there already finds the hit, but a nearer hit could still lie in a later
    # cell before it -- and none after: floor((x_hit - lo) / h) + 1 cells, one
    # sphere test in each.
    sc = S.make_scene([[0.0, 0.0, 0.0, 5.0]])
    gi = oracle.grid_info(sc, lam=lam)
    y, z = yz
    x_hit = -math.sqrt(25.0 - y * y - z * z)
    h = (gi["hi"][0] - gi["lo"][0]) / gi["dims"][0]
    expect = math.floor((x_hit - gi["lo"][0]) / h) + 1
    assert expect >= 2
    d = oracle.nearest_detail(sc, np.array([[-20.0, y, z]]), np.array([[1.0, 0.0, 0.0]]), mode="grid", lam=lam)
    assert d["id"][0] == 0 and d["t"][0] == pytest.approx(20.0 + x_hit, abs=1e-12)
    cells, sphere_tests, cylinder_tests = (int(c) for c in d["counters"])
    assert (cells, sphere_tests, cylinder_tests) == (expect, expect, 0)


@pytest.mark.parametrize("lam", [125.0, 1000.0, 8000.0])
def test_anyhit_walk_counts(oracle, lam):
    # The any-hit walk (AO and shadow rays) stops at the first test that hits.
    # One sphere listed in every cell of its box: a ray meeting it is done in
    # the cell where it enters the box (1 cell, 1 test); a ray through the box
    # that misses it walks every cell along x (n_x cells, one test each). A
    # tube along x, seen by a ray parallel to its axis inside its box, is
    # tested in every cell and never hit.
    sph = S.make_scene([[0.0, 0.0, 0.0, 5.0]])
    nx = oracle.grid_info(sph, lam=lam)["dims"][0]
    hit, cnt = oracle.anyhit(sph, np.array([[-20.0, 4.0, 0.3]]), np.array([[1.0, 0.0, 0.0]]), mode="grid", lam=lam)
    assert hit[0] and tuple(cnt) == (1, 1, 0)
    hit, cnt = oracle.anyhit(sph, np.array([[-20.0, 4.5, 4.5]]), np.array([[1.0, 0.0, 0.0]]), mode="grid", lam=lam)
    assert not hit[0] and tuple(cnt) == (nx, nx, 0)
    tube = S.make_scene(np.zeros((0, 4)), [[-5.0, 0.0, 0.0, 5.0, 0.0, 0.0, 1.0]])
    nx = oracle.grid_info(tube, lam=lam)["dims"][0]
    hit, cnt = oracle.anyhit(tube, np.array([[-20.0, 0.9, 0.9]]), np.array([[1.0, 0.0, 0.0]]), mode="grid", lam=lam)
    assert not hit[0] and tuple(cnt) == (nx, 0, nx)


@pytest.mark.parametrize("tmax", [math.inf, 3.0])
def test_anyhit_equals_brute_force_and_nearest(oracle, tmax):
    # grid and brute-force any-hit agree, and both say "hit" exactly when the
    # nearest hit lies in (0, tmax]
    sc = S.globule(200, 190, 10.0, seed=4)
    rng = np.random.default_rng(11)
    o = rng.uniform(-12.0, 12.0, (3000, 3))
    d = rng.normal(size=(3000, 3))
    hg, _ = oracle.anyhit(sc, o, d, mode="grid", lam=4.0, tmax=tmax)
    hb, _ = oracle.anyhit(sc, o, d, mode="brute", tmax=tmax)
    ids, ts, _, _ = oracle.nearest(sc, o, d, mode="brute")
    near = (ids != oracle.MISS) & (ts <= tmax)
    assert np.array_equal(hg, hb)
    assert np.array_equal(hb, near)
    assert 0.1 < hb.mean() < 0.9


def test_grid_reference_count(oracle):
    # every object is listed in exactly the cells its padded box overlaps
    sc = tiny_scene(4, n_sph=30, n_cyl=0)
    info = oracle.grid_info(sc, 1.0)
    lo, hi = info["lo"], info["hi"]
    dims = np.array(info["dims"])
    h = (hi - lo) / dims
    ext = (hi - lo).max()
    pad = 1e-5 * max(ext - 2 * 1e-5 * max(ext, 1.0), 1.0)
    refs = 0
    for s in sc.spheres.astype(np.float64):
        a = np.clip(np.floor((s[:3] - s[3] - pad - lo) / h), 0, dims - 1)
        b = np.clip(np.floor((s[:3] + s[3] + pad - lo) / h), 0, dims - 1)
        refs += int(np.prod(b - a + 1))
    assert refs == info["refs"]


def test_empty_scene_all_miss(oracle):
    sc = S.make_scene(np.zeros((0, 4)))
    o, d = random_rays(1, 50)
    for mode in ("brute", "grid"):
        ids, _, _, _ = oracle.nearest(sc, o, d, mode=mode)
        assert np.all(ids == oracle.MISS)
