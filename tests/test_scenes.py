"""The seeded input generator produces the stated workloads."""
import numpy as np

from paper_0801_1500_gb300 import scenes as S


def test_small_globule_recipe():
    sc = S.globule(2000, 1900, 25.0, seed=0)
    assert sc.spheres.shape == (2000, 4) and sc.cylinders.shape == (1900, 7)
    assert sc.spheres.dtype == np.float32 and sc.cylinders.dtype == np.float32
    r = sc.spheres[:, 3]
    assert r.min() >= 1.2 and r.max() <= 2.0
    assert np.all(np.linalg.norm(sc.spheres[:, :3].astype(np.float64), axis=1) <= 25.0 + 1e-4)
    bond = np.linalg.norm(sc.cylinders[:, 3:6].astype(np.float64) - sc.cylinders[:, 0:3], axis=1)
    assert np.allclose(bond, 3.8, atol=1e-4)
    assert np.all(sc.cylinders[:, 6] == np.float32(0.3))
    # each cylinder joins two consecutive atoms of one chain
    cen = {tuple(c) for c in sc.spheres[:, :3].tolist()}
    assert all(tuple(c) in cen for c in sc.cylinders[:, 0:3].tolist())
    assert sc.color_idx.shape == (3900,) and sc.color_idx.max() < 16


def test_paper_scene_counts_and_determinism():
    a = S.paper_scene(0)
    assert (a.n_spheres, a.n_cylinders) == (13500, 12818)
    assert a.n_objects == 26318
    b = S.paper_scene(0)
    assert np.array_equal(a.spheres, b.spheres) and np.array_equal(a.cylinders, b.cylinders)
    c = S.paper_scene(1)
    assert not np.array_equal(a.spheres, c.spheres)


def test_chain_lengths():
    ls = S.chain_lengths(13500, 12818)
    assert len(ls) == 682 and sum(ls) == 13500 and set(ls) == {19, 20}


def test_camera_aspect_and_orbit():
    sc = S.globule(200, 190, 10.0, seed=1)
    cam = S.ortho_camera(sc, 965, 1137)
    assert abs(cam.half_w / cam.half_h - 965 / 1137) < 1e-12
    for k in range(8):
        c = S.ortho_camera(sc, 512, 512, angle_deg=45.0 * k)
        d, r, u = np.array(c.dir), np.array(c.right), np.array(c.up)
        assert np.allclose([d @ d, r @ r, u @ u], 1) and abs(d @ r) < 1e-12 and abs(d @ u) < 1e-12
        assert np.allclose(np.cross(r, u), -d)


def test_traces():
    frames = S.orbit_frames(S.globule(200, 190, 10.0), 64)
    assert len(frames) == 64 and all(8 <= f["spp"] <= 32 for f in frames)
    assert {(f["width"], f["height"]) for f in frames} <= set(S.ORBIT_RESOLUTIONS)
    tr = S.poisson_trace(500, 200.0, 8, seed=0)
    gaps = np.diff([0.0] + [r["arrival_s"] for r in tr])
    assert abs(gaps.mean() - 1 / 200) < 0.2 / 200
    scenes = S.serving_scenes(3, 1000, 20000)
    assert [s.n_objects for s in scenes][0] >= 900 and scenes[-1].n_objects <= 21000


def test_md_trajectory_frames():
    base = S.globule(300, 285, 10.0, seed=2)
    traj = S.MDTrajectory(base, amplitude=0.3, period=16, spin_deg=3.0, seed=4)
    f0 = traj.frame(0)
    assert np.array_equal(f0.spheres, base.spheres) and np.array_equal(f0.cylinders, base.cylinders)
    pairs = S.bond_pairs(300, 285)
    assert pairs.shape == (285, 2)
    for k in (1, 5, 11, 35):
        f = traj.frame(k)
        # bonds follow their atoms; radii and colours stay
        assert np.array_equal(f.cylinders[:, 0:3], f.spheres[pairs[:, 0], :3])
        assert np.array_equal(f.cylinders[:, 3:6], f.spheres[pairs[:, 1], :3])
        assert np.array_equal(f.spheres[:, 3], base.spheres[:, 3])
        assert np.array_equal(f.cylinders[:, 6], base.cylinders[:, 6])
        # undo the spin: the thermal displacement is bounded by 2 sqrt(3) amplitude
        th = np.radians(3.0 * k)
        c = f.spheres[:, :3].astype(np.float64) - traj.centre
        x = np.cos(th) * c[:, 0] - np.sin(th) * c[:, 2]
        z = np.sin(th) * c[:, 0] + np.cos(th) * c[:, 2]
        un = np.stack([x, c[:, 1], z], axis=1) + traj.centre
        disp = np.linalg.norm(un - base.spheres[:, :3], axis=1)
        assert disp.max() <= 2.0 * np.sqrt(3.0) * 0.3 + 1e-4
        assert disp.max() > 0.05
    # periodic in the thermal part: frame `period` differs from frame 0 by the spin only
    assert np.array_equal(S.MDTrajectory(base, period=16, spin_deg=0.0, seed=4).frame(16).spheres.round(4),
                          base.spheres.round(4))
    assert np.array_equal(traj.frame(7).spheres, S.MDTrajectory(base, 0.3, 16, 3.0, 4).frame(7).spheres)
