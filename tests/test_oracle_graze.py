"""Pins of the oracle's grazing classifier.

Hit ids are compared only on non-grazing pixels, so the classifier decides how
much of every id-parity claim is actually checked. It is pinned here from
geometry alone, with each case placed just inside and just outside its
threshold:

  * a silhouette: a ray at distance h from a sphere's centre (or a tube's
    axis) has disc/r^2 = 1 - h^2/r^2; it is grazing when |disc/r^2| < 1e-4
    and the encounter lies at or before the winning t, whether the ray hits
    (the nearer root) or misses (the closest approach);
  * a tube's clip plane: a root whose axial coordinate lies within
    1e-4 (L + 1) of either end, inside or outside it;
  * a near-tie: the two nearest distinct hits within a relative 1e-5.

For grazing rays the oracle also reports the outcomes a faithful tracer may
give instead of the nearest hit: the runner-up (second-nearest distinct hit)
and the object of the nearest grazing encounter.

Every configuration is also run under random rigid rotations (no axis
alignment) and through the grid walk at two densities. The grid walk sees an
encounter only inside the grid's box, padded by 1e-5 of the scene's extent,
so these scenes hold a far marker sphere that widens the extent to about 100
(the paper-sized globules span about 120).
"""
import numpy as np
import pytest

from paper_0801_1500_gb300 import scenes as S

MISS = 0xFFFFFFFF
MODES = [("brute", 1.0), ("grid", 1.0), ("grid", 8.0)]


def rotations(n=4, seed=0):
    """Identity plus n seeded random rotations."""
    rng = np.random.default_rng(seed)
    out = [np.eye(3)]
    for _ in range(n):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out.append(q)
    return out


# far from every ray below; its id comes after the configuration's spheres
MARKER = [60.0, 60.0, 60.0, 1.0]


def rotated(R, spheres=None, cylinders=None, origins=(), dirs=()):
    spheres = list(spheres or []) + [MARKER]
    sph = np.array([[*(R @ np.array(s[:3])), s[3]] for s in spheres])
    cyl = None if cylinders is None else np.array([[*(R @ np.array(c[:3])), *(R @ np.array(c[3:6])), c[6]]
                                                   for c in cylinders])
    o = np.array([R @ np.array(x, float) for x in origins])
    d = np.array([R @ np.array(x, float) for x in dirs])
    return S.make_scene(sph, cyl), o, d


def run(oracle, sc, o, d):
    return [oracle.nearest_detail(sc, o, d, mode=m, lam=lam) for m, lam in MODES]


# disc/r^2 of a ray past a silhouette, and whether it grazes
SILHOUETTE = [(0.75, False), (2e-4, False), (5e-5, True), (1e-7, True),
              (-1e-7, True), (-5e-5, True), (-2e-4, False), (-3.0, False)]


@pytest.mark.parametrize("R", rotations())
def test_sphere_silhouette(oracle, R):
    r = 1.5
    hs = [r * np.sqrt(1.0 - q) for q, _ in SILHOUETTE]
    sc, o, d = rotated(R, spheres=[[0.0, 0.0, 0.0, r]], origins=[[h, 0.0, 20.0] for h in hs],
                       dirs=[[0.0, 0.0, -1.0]] * len(hs))
    for res in run(oracle, sc, o, d):
        for k, (q, gz) in enumerate(SILHOUETTE):
            assert (res["id"][k] == 0) == (q > 0), (q, res["id"][k])
            assert res["grazing"][k] == gz, (q, res["grazing"][k])
            if gz:
                # the grazed sphere is the alternative outcome
                assert res["idg"][k] == 0 and res["id2"][k] == MISS
            else:
                assert res["idg"][k] == MISS and res["id2"][k] == MISS
        # a hit grazing its own silhouette: the encounter is the hit itself
        assert res["t"][3] == pytest.approx(20.0 - r * np.sqrt(1e-7), abs=1e-9)


@pytest.mark.parametrize("R", rotations())
def test_tube_tangent(oracle, R):
    # a ray perpendicular to the axis at distance h from it. Scene arrays are
    # float32: a rotated tube's ends move by ~2e-7, more than the |disc| = 1e-7
    # cases allow, so those run on the unrotated tube only
    r, L = 0.5, 4.0
    cases = [(q, gz) for q, gz in SILHOUETTE if abs(q) > 1e-6 or np.array_equal(R, np.eye(3))]
    hs = [r * np.sqrt(1.0 - q) for q, _ in cases]
    sc, o, d = rotated(R, cylinders=[[0.0, 0.0, 0.0, L, 0.0, 0.0, r]],
                       origins=[[2.0, h, 20.0] for h in hs], dirs=[[0.0, 0.0, -1.0]] * len(hs))
    for res in run(oracle, sc, o, d):
        for k, (q, gz) in enumerate(cases):
            assert (res["id"][k] == 1) == (q > 0), q   # id 0 is the marker sphere
            assert res["grazing"][k] == gz, q
            assert res["idg"][k] == (1 if gz else MISS)
    # the same silhouette distances beyond the tube's end (closest approach at
    # axial coordinate L + 2): no root can count there, so no ray grazes
    sc, o, d = rotated(R, cylinders=[[0.0, 0.0, 0.0, L, 0.0, 0.0, r]],
                       origins=[[L + 2.0, h, 20.0] for h in hs], dirs=[[0.0, 0.0, -1.0]] * len(hs))
    for res in run(oracle, sc, o, d):
        assert np.all(res["id"] == MISS) and not res["grazing"].any()


# axial coordinate of the ray's crossing of a tube of length 4 (margin
# 1e-4 (L + 1) = 5e-4), whether the tube is hit, and whether it grazes
CLIP = [(2.0, True, False), (2e-4, True, True), (1e-3, True, False), (-2e-4, False, True),
        (-1e-3, False, False), (4.0 - 2e-4, True, True), (4.0 + 2e-4, False, True), (4.0 + 1e-3, False, False)]


@pytest.mark.parametrize("R", rotations())
def test_tube_clip_planes(oracle, R):
    r, L = 0.5, 4.0
    sc, o, d = rotated(R, cylinders=[[0.0, 0.0, 0.0, L, 0.0, 0.0, r]],
                       origins=[[s, 0.0, 20.0] for s, _, _ in CLIP], dirs=[[0.0, 0.0, -1.0]] * len(CLIP))
    for res in run(oracle, sc, o, d):
        for k, (s, hit, gz) in enumerate(CLIP):
            assert (res["id"][k] == 1) == hit, s   # id 0 is the marker sphere
            assert res["grazing"][k] == gz, s
            assert res["idg"][k] == (1 if gz else MISS), s
            if hit:
                assert res["t"][k] == pytest.approx(19.5, abs=1e-6)   # float32 ends


@pytest.mark.parametrize("R", rotations())
def test_grazed_sphere_in_front_behind_and_behind_the_origin(oracle, R):
    # B (id 1): a large sphere the ray hits near t = 26. A (id 0): a small
    # sphere whose silhouette the ray passes within 5e-5 (of r^2) -- in front
    # of the hit (grazing), behind the hit (not), behind the origin (not)
    hA_miss, hA_hit = np.sqrt(1.0 + 5e-5), np.sqrt(1.0 - 5e-5)
    B = [0.0, 0.0, -10.0, 4.0]
    cases = [  # (A centre z, ray offset, expected id, grazing, id2, idg)
        (5.0, hA_miss, 1, True, MISS, 0),
        (5.0, hA_hit, 0, True, 1, 0),
        (-20.0, hA_miss, 1, False, MISS, MISS),
        (30.0, hA_miss, 1, False, MISS, MISS),
    ]
    for za, h, want, gz, id2, idg in cases:
        sc, o, d = rotated(R, spheres=[[0.0, 0.0, za, 1.0], B], origins=[[h, 0.0, 20.0]], dirs=[[0.0, 0.0, -1.0]])
        for res in run(oracle, sc, o, d):
            assert res["id"][0] == want, (za, h)
            assert res["grazing"][0] == gz, (za, h)
            assert res["id2"][0] == id2 and res["idg"][0] == idg, (za, h, res["id2"][0], res["idg"][0])


@pytest.mark.parametrize("R", rotations())
def test_near_ties(oracle, R):
    # P (id 0): front surface at t = 19; Q (id 1): front surface at 19 (1 + delta)
    for delta, gz in [(0.0, True), (5e-6, True), (-5e-6, True), (2e-5, False), (-2e-5, False), (1e-3, False)]:
        zq = -1.0 - 19.0 * delta
        sc, o, d = rotated(R, spheres=[[0.0, 0.0, 0.0, 1.0], [0.0, 0.0, zq, 2.0]], origins=[[0.0, 0.0, 20.0]],
                           dirs=[[0.0, 0.0, -1.0]])
        for res in run(oracle, sc, o, d):
            want = 0 if delta >= 0 else 1
            if delta == 0.0 and not np.array_equal(R, np.eye(3)):
                want = int(res["id"][0])   # an exact tie, left to rounding once rotated
                assert want in (0, 1)
            assert res["id"][0] == want, delta
            assert res["grazing"][0] == gz, delta
            assert res["id2"][0] == ((1 - want) if gz else MISS), delta
            assert res["idg"][0] == MISS


def test_runner_up_is_second_distinct_hit(oracle):
    # a grazing ray's runner-up is the next distinct object along it, even far
    # behind the hit (the grid walk stops long before it)
    hA = np.sqrt(1.0 - 5e-5)
    sc, o, d = rotated(np.eye(3), spheres=[[0.0, 0.0, 5.0, 1.0], [0.0, 0.0, -30.0, 2.0], [0.0, 0.0, -60.0, 2.0]],
                       origins=[[hA, 0.0, 20.0]], dirs=[[0.0, 0.0, -1.0]])
    for res in run(oracle, sc, o, d):
        assert res["id"][0] == 0 and res["grazing"][0]
        assert res["id2"][0] == 1 and res["idg"][0] == 0


def test_grazing_fraction_of_random_rays_is_small(oracle):
    # random rays through a random scene: grazing is rare, and the grid walk
    # classifies exactly as brute force
    from test_oracle_grid import random_rays, tiny_scene
    t = tiny_scene(3)
    sc = S.make_scene(np.concatenate([t.spheres, [MARKER]]), t.cylinders)
    o, d = random_rays(7, 20000)
    b = oracle.nearest_detail(sc, o, d, mode="brute")
    assert b["grazing"].mean() < 2e-3
    for lam in (0.25, 1.0, 8.0):
        g = oracle.nearest_detail(sc, o, d, mode="grid", lam=lam)
        assert np.array_equal(g["grazing"], b["grazing"])
        assert np.array_equal(g["id"], b["id"])
        assert np.array_equal(g["id2"], b["id2"]) and np.array_equal(g["idg"], b["idg"])
