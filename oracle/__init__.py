"""FP64 CPU oracle of the molecular AO ray tracer (ctypes wrapper).

TEST INFRASTRUCTURE: imported only by the test suite, the package smoke check
and the benchmark's CPU-baseline leg. It shares no code with the CUDA library
and imports nothing from it; scene/camera/light/parameter objects are read by
attribute name (duck typing) so the same seeded inputs can be handed to both.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None
MISS = 0xFFFFFFFF


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB lets the test suite load a deliberately mutated build
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32, u32, u64, f64 = C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_ao_uniforms.argtypes = [u32, u32, u32, u64, P, P]
        L.oracle_onb.argtypes = [P, P, P]
        L.oracle_cosine_dir.argtypes = [P, f64, f64, P]
        L.oracle_hit_sphere.argtypes = [P, P, P, f64, f64, f64, P, P]
        L.oracle_hit_cylinder.argtypes = [P, P, P, P, f64, f64, f64, P, P]
        L.oracle_nearest.argtypes = [i64, P, i64, P, i32, f64, i64, P, P, f64, f64, P, P, P, P, P, P]
        L.oracle_anyhit.argtypes = [i64, P, i64, P, i32, f64, i64, P, P, f64, P, P]
        L.oracle_grid_walk.argtypes = [i64, P, i64, P, f64, P, P, f64, f64, i64, P, P]
        L.oracle_grid_info.argtypes = [i64, P, i64, P, f64, P, P, P]
        L.oracle_ao_probe.argtypes = [i64, P, i64, P, i32, f64, i64, P, P, i32, u64, u32, f64, f64, P, i32]
        L.oracle_render.argtypes = [i64, P, i64, P, P, P, i32, P, i32, i32, P, P, i32, P,
                                    i32, u64, u32, i32, f64, i64, P, P, P, P, P, P, P, P, P, i32]
        L.oracle_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


MODES = {"brute": 0, "grid": 1}


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, np.uint32).reshape(2))
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def ao_uniforms(index, sample, frame, seed):
    u1, u2 = C.c_double(), C.c_double()
    lib().oracle_ao_uniforms(index, sample, frame, seed, C.byref(u1), C.byref(u2))
    return u1.value, u2.value


def onb(n):
    n = _f64(n, 3)
    b1, b2 = np.zeros(3), np.zeros(3)
    lib().oracle_onb(_p(n), _p(b1), _p(b2))
    return b1, b2


def cosine_dir(n, u1, u2):
    n = _f64(n, 3)
    d = np.zeros(3)
    lib().oracle_cosine_dir(_p(n), float(u1), float(u2), _p(d))
    return d


class _Graze(C.Structure):
    _fields_ = [("disc_rel", C.c_double), ("t_close", C.c_double), ("t_near", C.c_double),
                ("s_out", C.c_double), ("end_mrg", C.c_double * 2), ("t_end", C.c_double * 2)]


def hit_sphere(o, d, c, r, tmin=0.0, tmax=math.inf):
    """Nearest root in (tmin, tmax] of a unit-direction ray; None on a miss."""
    o, d, c = _f64(o, 3), _f64(d, 3), _f64(c, 3)
    t = C.c_double()
    g = _Graze()
    hit = lib().oracle_hit_sphere(_p(o), _p(d), _p(c), float(r), float(tmin), float(tmax), C.byref(t), C.byref(g))
    return (t.value if hit else None), g.disc_rel


def hit_cylinder(o, d, p0, p1, r, tmin=0.0, tmax=math.inf):
    o, d, p0, p1 = _f64(o, 3), _f64(d, 3), _f64(p0, 3), _f64(p1, 3)
    t = C.c_double()
    g = _Graze()
    hit = lib().oracle_hit_cylinder(_p(o), _p(d), _p(p0), _p(p1), float(r), float(tmin), float(tmax),
                                    C.byref(t), C.byref(g))
    return (t.value if hit else None), g.disc_rel


# ---------------------------------------------------------------- scenes

def _scene_arrays(scene):
    sph = _f64(scene.spheres, (-1, 4))
    cyl = _f64(scene.cylinders, (-1, 7))
    col = np.ascontiguousarray(np.asarray(scene.color_idx, np.uint32))
    pal = _f64(scene.palette, (-1, 3))
    return sph, cyl, col, pal


def nearest_detail(scene, orig, dirs, mode="brute", lam=1.0, tmin=0.0, tmax=math.inf):
    """Nearest hits of explicit rays (directions are normalised), as a dict:
    id, t, grazing; for grazing rays id2 (the runner-up: second-nearest
    distinct hit) and idg (the object of the nearest grazing encounter), MISS
    where there is none and on non-grazing rays; counters (cells, sphere
    tests, cylinder tests)."""
    sph, cyl, _, _ = _scene_arrays(scene)
    o = _f64(orig, (-1, 3))
    d = _f64(dirs, (-1, 3))
    d = np.ascontiguousarray(d / np.linalg.norm(d, axis=1, keepdims=True))
    n = o.shape[0]
    ids = np.zeros(n, np.uint32)
    ts = np.zeros(n)
    gz = np.zeros(n, np.uint8)
    id2 = np.zeros(n, np.uint32)
    idg = np.zeros(n, np.uint32)
    cnt = np.zeros(3, np.int64)
    rc = lib().oracle_nearest(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), MODES[mode], float(lam), n,
                              _p(o), _p(d), float(tmin), float(tmax), _p(ids), _p(ts), _p(gz), _p(id2), _p(idg),
                              _p(cnt))
    if rc:
        raise RuntimeError("oracle_nearest failed")
    return dict(id=ids, t=ts, grazing=gz.astype(bool), id2=id2, idg=idg, counters=cnt)


def anyhit(scene, orig, dirs, mode="brute", lam=1.0, tmax=math.inf):
    """Any hit in (0, tmax] of explicit rays (directions are normalised), as
    (hit bool per ray, counters: cells, sphere tests, cylinder tests)."""
    sph, cyl, _, _ = _scene_arrays(scene)
    o = _f64(orig, (-1, 3))
    d = _f64(dirs, (-1, 3))
    d = np.ascontiguousarray(d / np.linalg.norm(d, axis=1, keepdims=True))
    n = o.shape[0]
    hit = np.zeros(n, np.uint8)
    cnt = np.zeros(3, np.int64)
    rc = lib().oracle_anyhit(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), MODES[mode], float(lam), n, _p(o), _p(d),
                             float(tmax), _p(hit), _p(cnt))
    if rc:
        raise RuntimeError("oracle_anyhit failed")
    return hit.astype(bool), cnt


def nearest(scene, orig, dirs, mode="brute", lam=1.0, tmin=0.0, tmax=math.inf):
    """Nearest hit (id, t, grazing flag, counters) of explicit rays; directions are normalised."""
    r = nearest_detail(scene, orig, dirs, mode=mode, lam=lam, tmin=tmin, tmax=tmax)
    return r["id"], r["t"], r["grazing"], r["counters"]


def grid_walk(scene, o, d, lam=1.0, tmin=0.0, tmax=math.inf, max_out=1 << 16):
    sph, cyl, _, _ = _scene_arrays(scene)
    o, d = _f64(o, 3), _f64(d, 3)
    d = d / np.linalg.norm(d)
    out = np.zeros(max_out, np.int64)
    dims = np.zeros(3, np.int32)
    n = lib().oracle_grid_walk(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), float(lam), _p(o), _p(d),
                               float(tmin), float(tmax), max_out, _p(out), _p(dims))
    if n < 0:
        raise RuntimeError("oracle_grid_walk failed")
    return out[:min(n, max_out)], tuple(int(x) for x in dims)


def grid_info(scene, lam=1.0):
    sph, cyl, _, _ = _scene_arrays(scene)
    lohi = np.zeros(6)
    dims = np.zeros(3, np.int32)
    refs = np.zeros(1, np.int64)
    if lib().oracle_grid_info(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), float(lam), _p(lohi), _p(dims), _p(refs)):
        raise RuntimeError("oracle_grid_info failed")
    return dict(lo=lohi[:3].copy(), hi=lohi[3:].copy(), dims=tuple(int(x) for x in dims), refs=int(refs[0]))


def ao_probe(scene, pts, nrm, spp, seed=0, frame=0, eps=1e-3, maxdist=math.inf, mode="grid", lam=1.0,
             threads=0):
    sph, cyl, _, _ = _scene_arrays(scene)
    p = _f64(pts, (-1, 3))
    n = _f64(nrm, (-1, 3))
    out = np.zeros(p.shape[0])
    rc = lib().oracle_ao_probe(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), MODES[mode], float(lam),
                               p.shape[0], _p(p), _p(n), int(spp), int(seed), int(frame), float(eps),
                               float(maxdist), _p(out), int(threads))
    if rc:
        raise RuntimeError("oracle_ao_probe failed")
    return out


def camera_vector(cam):
    """Flatten a camera object: kind, eye, dir, up, right, half_w, half_h,
    sub-pixel grid side m (``aa``, default 1)."""
    v = np.zeros(16)
    v[0] = float(cam.kind)
    v[1:4] = cam.eye
    v[4:7] = cam.dir
    v[7:10] = cam.up
    v[10:13] = cam.right
    v[13] = cam.half_w
    v[14] = cam.half_h
    v[15] = float(max(1, int(getattr(cam, "aa", 1) or 1)))
    return v


def shade_vector(lights, params):
    sp = np.zeros(12)
    sp[0] = lights.scale
    sp[1] = lights.skylight
    sp[2] = params.k_ao
    sp[3] = params.k_d
    sp[4] = params.k_s
    sp[5] = params.phong_exp
    sp[6] = params.eps
    sp[7] = params.ao_maxdist
    sp[8:11] = params.background
    sp[11] = 1.0 if getattr(params, "shadows", False) else 0.0
    return sp


COUNTER_NAMES = ["primary_rays", "ao_rays", "hit_pixels", "primary_cells", "primary_sphere_tests",
                 "primary_cylinder_tests", "ao_cells", "ao_sphere_tests", "ao_cylinder_tests", "ao_unoccluded"]


def render(scene, camera, width, height, lights, params, pixels=None, mode="grid", lam=1.0, threads=0,
           spp=None):
    """Render the listed pixel indices (j*W + i), or the whole frame.

    Returns a dict with rgb [n,3] float64 per pixel and, per sub-sample
    (n m^2 entries, pixel-major, then sub-row b, then sub-column a; m = the
    camera's sub-pixel grid side, 1 without supersampling): id uint32
    (0xFFFFFFFF = miss), t, vis (unoccluded AO samples), grazing bool, and for
    grazing sub-samples id2 (the runner-up) and idg (the object of the
    nearest grazing encounter), MISS where there is none; and a counters dict.
    """
    sph, cyl, col, pal = _scene_arrays(scene)
    cam = camera_vector(camera)
    ldir = _f64(lights.dirs, (-1, 3))
    lI = _f64(lights.intensity, (-1,))
    sp = shade_vector(lights, params)
    spp = params.ao_samples if spp is None else spp
    if pixels is None:
        npix = int(width) * int(height)
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, np.int64))
        npix = pix.shape[0]
    nsub = npix * int(cam[15]) ** 2
    rgb = np.zeros((npix, 3))
    ids = np.zeros(nsub, np.uint32)
    ts = np.zeros(nsub)
    vis = np.zeros(nsub, np.int32)
    gz = np.zeros(nsub, np.uint8)
    id2 = np.zeros(nsub, np.uint32)
    idg = np.zeros(nsub, np.uint32)
    cnt = np.zeros(16, np.int64)
    rc = lib().oracle_render(sph.shape[0], _p(sph), cyl.shape[0], _p(cyl), _p(col), _p(pal), pal.shape[0],
                             _p(cam), int(width), int(height), _p(ldir), _p(lI), ldir.shape[0], _p(sp),
                             int(spp), int(params.seed), int(params.frame), MODES[mode], float(lam),
                             npix, _p(pix), _p(rgb), _p(ids), _p(ts), _p(vis), _p(gz), _p(id2), _p(idg), _p(cnt),
                             int(threads))
    if rc:
        raise RuntimeError(f"oracle_render failed ({rc})")
    return dict(rgb=rgb, id=ids, t=ts, vis=vis, grazing=gz.astype(bool), id2=id2, idg=idg,
                counters={k: int(cnt[i]) for i, k in enumerate(COUNTER_NAMES)})
