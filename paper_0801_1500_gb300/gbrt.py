"""Thin ctypes binding of libgbrt (include/gbrt.h).

Functions keep the C names and only marshal arguments: torch CUDA tensors and
numpy arrays become pointers, dataclasses from ``scenes`` become the C structs.
Every step of the render runs in the library's CUDA kernels; there is no CPU
path. Importing this module loads ``libgbrt.so`` and raises if it is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

# GBRT_LIB_VARIANT=checked loads the checked build (indices tested against
# their buffers; see build.py)
LIB_PATH = _build.LIB_CHECKED if os.environ.get("GBRT_LIB_VARIANT") == "checked" else _build.LIB

OK, EINVAL, ENOMEM, EDEVICE, ETIMEDOUT, ETRAVERSAL, ECAPACITY, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
DEVICE_PTRS, HOST_PTRS, BATCH_GRAPH, HOST_ASYNC = 0, 1, 2, 4
FP32, FP64 = 0, 1
CAMERA_ORTHO, CAMERA_PINHOLE = 0, 1
MAX_LIGHTS = 8
MAX_AA = 4          # largest sub-pixel grid side (camera aa)
MISS = 0xFFFFFFFF


class GbrtError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class gbrt_camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("aa", C.c_int32), ("eye", C.c_double * 3), ("dir", C.c_double * 3),
                ("up", C.c_double * 3), ("right", C.c_double * 3), ("half_w", C.c_double), ("half_h", C.c_double)]


class gbrt_lights(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved", C.c_int32), ("dir", (C.c_double * 3) * MAX_LIGHTS),
                ("intensity", C.c_double * MAX_LIGHTS), ("scale", C.c_double), ("skylight", C.c_double)]


class gbrt_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("out_flags", C.c_int32), ("seed", C.c_uint64), ("frame", C.c_uint32),
                ("shadows", C.c_int32), ("eps", C.c_double), ("ao_maxdist", C.c_double), ("k_ao", C.c_double),
                ("k_d", C.c_double), ("k_s", C.c_double), ("phong_exp", C.c_double),
                ("background", C.c_double * 3)]


class gbrt_render_item(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("grid", C.c_void_p), ("camera", gbrt_camera), ("width", C.c_int32),
                ("height", C.c_int32), ("ao_samples", C.c_int32), ("reserved", C.c_int32),
                ("row_begin", C.c_int32), ("row_end", C.c_int32),
                ("lights", gbrt_lights), ("params", gbrt_params), ("out_rgb", C.c_void_p),
                ("out_hit_ids", C.c_void_p), ("out_ao_visible", C.c_void_p)]


class gbrt_tuning(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("block", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("refill", C.c_int32), ("reserved", C.c_int32 * 3)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    P, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "gbrt_version": ([], C.c_int),
        "gbrt_strerror": ([C.c_int], C.c_char_p),
        "gbrt_create": ([P, C.c_int, P], C.c_int),
        "gbrt_set_stream": ([P, P], C.c_int),
        "gbrt_sync": ([P], C.c_int),
        "gbrt_destroy": ([P], C.c_int),
        "gbrt_scene_upload": ([P, P, i64, P, i64, P, P, i32, C.c_int, P], C.c_int),
        "gbrt_scene_info": ([P, P, P, P], C.c_int),
        "gbrt_scene_free": ([P, P], C.c_int),
        "gbrt_grid_build": ([P, P, f32, P], C.c_int),
        "gbrt_grid_info": ([P, P, P, P, P, P], C.c_int),
        "gbrt_grid_free": ([P, P], C.c_int),
        "gbrt_scene_update": ([P, P, P, P, C.c_int], C.c_int),
        "gbrt_microbench": ([P, C.c_int, C.POINTER(C.c_double)], C.c_int),
        "gbrt_grid_rebuild": ([P, P, P], C.c_int),
        "gbrt_render": ([P, P, P, C.POINTER(gbrt_camera), i32, i32, i32, C.POINTER(gbrt_lights),
                         C.POINTER(gbrt_params), P, P, P], C.c_int),
        "gbrt_render_batch": ([P, C.POINTER(gbrt_render_item), i32, C.c_int], C.c_int),
        "gbrt_ao_probe": ([P, P, P, P, P, i64, i32, C.POINTER(gbrt_params), P], C.c_int),
        "gbrt_philox4x32_10": ([P, P, P, i64, P], C.c_int),
        "gbrt_set_tuning": ([P, C.POINTER(gbrt_tuning)], C.c_int),
        "gbrt_get_tuning": ([P, C.POINTER(gbrt_tuning)], C.c_int),
        "gbrt_launch_count": ([P], C.c_int64),
        "gbrt_set_profiling": ([P, C.c_int], C.c_int),
        "gbrt_phase_times": ([P, P], C.c_int),
        "gbrt_render_noalloc": ([P, P, C.POINTER(gbrt_camera), i32, i32, i32, C.POINTER(gbrt_lights),
                                 C.POINTER(gbrt_params), P, P, P, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


def strerror(code: int) -> str:
    return lib.gbrt_strerror(int(code)).decode()


def _check(code, where):
    if code != OK:
        raise GbrtError(code, where)
    return code


def ptr(x):
    """Address of a torch tensor, numpy array or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take the address of {type(x)}")


def _buf(x, nbytes, host, where):
    """Address of an argument buffer after checking that it is dense, in the
    expected memory (host or device) and at least ``nbytes`` long; None passes
    through and a raw integer address is taken as given. A mismatch raises
    GbrtError(EINVAL) before the library is called."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous() or bool(x.is_cuda) == bool(host):
            raise GbrtError(EINVAL, where)
        size = x.numel() * x.element_size()
    elif isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or not host:
            raise GbrtError(EINVAL, where)
        size = x.nbytes
    else:
        raise TypeError(f"{where}: cannot take the address of {type(x)}")
    if size < nbytes:
        raise GbrtError(EINVAL, where)
    return ptr(x)


def _frame_bytes(camera, width, height, params):
    """Bytes of a render's colour output and of each per-sub-sample output."""
    m = max(1, int(camera.aa))
    px = max(0, int(width)) * max(0, int(height))
    return px * 3 * (8 if int(params.precision) == FP64 else 4), px * m * m * 4


# ------------------------------------------------------------ struct builders

def make_camera(cam) -> gbrt_camera:
    c = gbrt_camera()
    c.kind = int(cam.kind)
    c.aa = int(getattr(cam, "aa", 1) or 1)
    for k in range(3):
        c.eye[k], c.dir[k], c.up[k], c.right[k] = cam.eye[k], cam.dir[k], cam.up[k], cam.right[k]
    c.half_w, c.half_h = float(cam.half_w), float(cam.half_h)
    return c


def make_lights(lights) -> gbrt_lights:
    L = gbrt_lights()
    L.n = len(lights.dirs)
    for l, (d, i) in enumerate(zip(lights.dirs, lights.intensity)):
        for k in range(3):
            L.dir[l][k] = float(d[k])
        L.intensity[l] = float(i)
    L.scale = float(lights.scale)
    L.skylight = float(lights.skylight)
    return L


def make_params(p, precision=None, out_flags=0) -> gbrt_params:
    q = gbrt_params()
    q.precision = int(p.precision if precision is None else precision)
    q.out_flags = int(out_flags)
    q.seed = int(p.seed)
    q.frame = int(p.frame)
    q.shadows = 1 if getattr(p, "shadows", False) else 0
    q.eps = float(p.eps)
    q.ao_maxdist = float(p.ao_maxdist)
    q.k_ao, q.k_d, q.k_s, q.phong_exp = float(p.k_ao), float(p.k_d), float(p.k_s), float(p.phong_exp)
    for k in range(3):
        q.background[k] = float(p.background[k])
    return q


# ------------------------------------------------------------ C calls

def gbrt_version() -> int:
    return lib.gbrt_version()


def gbrt_create(device: int = 0, stream=None):
    h = C.c_void_p()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.gbrt_create(C.byref(h), int(device), s), "gbrt_create")
    return h.value


def gbrt_set_stream(ctx, stream):
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return _check(lib.gbrt_set_stream(ctx, s), "gbrt_set_stream")


def gbrt_sync(ctx, check=True):
    rc = lib.gbrt_sync(ctx)
    return _check(rc, "gbrt_sync") if check else rc


def gbrt_destroy(ctx):
    return _check(lib.gbrt_destroy(ctx), "gbrt_destroy")


def gbrt_scene_upload(ctx, spheres, cylinders, color_idx, palette, flags=None):
    """Arrays: torch CUDA tensors (device) or numpy arrays (host, flags = HOST_PTRS)."""
    if flags is None:
        flags = HOST_PTRS if isinstance(spheres, np.ndarray) else DEVICE_PTRS
    host = flags == HOST_PTRS
    if host:
        spheres = np.ascontiguousarray(spheres, np.float32)
        cylinders = np.ascontiguousarray(cylinders, np.float32)
        color_idx = np.ascontiguousarray(color_idx, np.uint32)
        palette = np.ascontiguousarray(palette, np.float32)
    S, Cn, K = int(spheres.shape[0]), int(cylinders.shape[0]), int(palette.shape[0])
    w = "gbrt_scene_upload"
    h = C.c_void_p()
    rc = lib.gbrt_scene_upload(ctx, _buf(spheres, 16 * S, host, w), S, _buf(cylinders, 28 * Cn, host, w), Cn,
                               _buf(color_idx, 4 * (S + Cn), host, w), _buf(palette, 12 * K, host, w), K,
                               int(flags), C.byref(h))
    _check(rc, "gbrt_scene_upload")
    return h.value


def gbrt_scene_info(scene):
    s, c, b = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib.gbrt_scene_info(scene, C.byref(s), C.byref(c), C.byref(b)), "gbrt_scene_info")
    return dict(n_spheres=s.value, n_cylinders=c.value, device_bytes=b.value)


def gbrt_scene_free(ctx, scene):
    return _check(lib.gbrt_scene_free(ctx, scene), "gbrt_scene_free")


def gbrt_grid_build(ctx, scene, lam=0.0):
    h = C.c_void_p()
    _check(lib.gbrt_grid_build(ctx, scene, float(lam), C.byref(h)), "gbrt_grid_build")
    return h.value


def gbrt_grid_info(grid):
    dims = (C.c_int32 * 3)()
    lo = (C.c_float * 3)()
    hi = (C.c_float * 3)()
    refs, nbytes = C.c_int64(), C.c_int64()
    _check(lib.gbrt_grid_info(grid, dims, lo, hi, C.byref(refs), C.byref(nbytes)), "gbrt_grid_info")
    return dict(dims=tuple(dims), lo=tuple(lo), hi=tuple(hi), refs=refs.value, device_bytes=nbytes.value)


def gbrt_grid_free(ctx, grid):
    return _check(lib.gbrt_grid_free(ctx, grid), "gbrt_grid_free")


def gbrt_scene_update(ctx, scene, spheres, cylinders, flags=None):
    """New geometry for a resident scene (same counts): torch CUDA tensors or
    numpy arrays (host; pinned ones are read asynchronously)."""
    if flags is None:
        flags = HOST_PTRS if isinstance(spheres, np.ndarray) else DEVICE_PTRS
    host = flags == HOST_PTRS
    if host:
        if not (isinstance(spheres, np.ndarray) and spheres.dtype == np.float32 and spheres.flags.c_contiguous):
            spheres = np.ascontiguousarray(spheres, np.float32)
        if not (isinstance(cylinders, np.ndarray) and cylinders.dtype == np.float32
                and cylinders.flags.c_contiguous):
            cylinders = np.ascontiguousarray(cylinders, np.float32)
    info = gbrt_scene_info(scene)
    w = "gbrt_scene_update"
    return _check(lib.gbrt_scene_update(ctx, scene, _buf(spheres, 16 * info["n_spheres"], host, w),
                                        _buf(cylinders, 28 * info["n_cylinders"], host, w), int(flags)), w)


MB_FP32_FMA, MB_FP64_FMA, MB_L2_READ = 0, 1, 2


def gbrt_microbench(ctx, kind):
    """FMA rate (TFLOP/s) or L2 read bandwidth (GB/s) of the context's GPU."""
    v = C.c_double()
    _check(lib.gbrt_microbench(ctx, int(kind), C.byref(v)), "gbrt_microbench")
    return v.value


def gbrt_grid_rebuild(ctx, grid, scene):
    return _check(lib.gbrt_grid_rebuild(ctx, grid, scene), "gbrt_grid_rebuild")


def gbrt_render(ctx, scene, grid, camera, width, height, ao_samples, lights, params, out_rgb, out_hit_ids=None,
                out_ao_visible=None):
    """camera/lights/params: C structs (make_*) or the ``scenes`` dataclasses."""
    cam = camera if isinstance(camera, gbrt_camera) else make_camera(camera)
    li = lights if isinstance(lights, gbrt_lights) else make_lights(lights)
    pa = params if isinstance(params, gbrt_params) else make_params(params)
    host = bool(pa.out_flags & HOST_PTRS)
    rgb_b, px_b = _frame_bytes(cam, width, height, pa)
    w = "gbrt_render"
    rc = lib.gbrt_render(ctx, scene, grid, C.byref(cam), int(width), int(height), int(ao_samples), C.byref(li),
                         C.byref(pa), _buf(out_rgb, rgb_b, host, w), _buf(out_hit_ids, px_b, host, w),
                         _buf(out_ao_visible, px_b, host, w))
    return _check(rc, w)


def gbrt_render_batch(ctx, items, flags=0):
    arr = (gbrt_render_item * len(items))(*items)
    return _check(lib.gbrt_render_batch(ctx, arr, len(items), int(flags)), "gbrt_render_batch")


NOALLOC_MAX_PIXELS = 65536


def gbrt_render_noalloc(scene, grid, camera, width, height, ao_samples, lights, params, out_rgb,
                        out_hit_ids=None, out_ao_visible=None, stream=None):
    """Render without any allocation (fixed in-library scratch, frames up to
    NOALLOC_MAX_PIXELS pixels); asynchronous on ``stream`` (a torch stream,
    a raw handle or None for the legacy default stream)."""
    cam = camera if isinstance(camera, gbrt_camera) else make_camera(camera)
    li = lights if isinstance(lights, gbrt_lights) else make_lights(lights)
    pa = params if isinstance(params, gbrt_params) else make_params(params)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    rgb_b, px_b = _frame_bytes(cam, width, height, pa)
    w = "gbrt_render_noalloc"
    rc = lib.gbrt_render_noalloc(scene, grid, C.byref(cam), int(width), int(height), int(ao_samples), C.byref(li),
                                 C.byref(pa), _buf(out_rgb, rgb_b, False, w), _buf(out_hit_ids, px_b, False, w),
                                 _buf(out_ao_visible, px_b, False, w), s)
    return _check(rc, w)


def gbrt_ao_probe(ctx, scene, grid, pts, nrm, ao_samples, params, out_visibility):
    pa = params if isinstance(params, gbrt_params) else make_params(params)
    n = int(pts.shape[0])
    w = "gbrt_ao_probe"
    rc = lib.gbrt_ao_probe(ctx, scene, grid, _buf(pts, 24 * n, False, w), _buf(nrm, 24 * n, False, w), n,
                           int(ao_samples), C.byref(pa), _buf(out_visibility, 4 * n, False, w))
    return _check(rc, w)


def gbrt_philox4x32_10(ctx, ctr, key, out):
    n = int(ctr.shape[0])
    w = "gbrt_philox4x32_10"
    return _check(lib.gbrt_philox4x32_10(ctx, _buf(ctr, 16 * n, False, w), _buf(key, 8 * n, False, w), n,
                                         _buf(out, 16 * n, False, w)), w)


def gbrt_set_tuning(ctx, tile_w=8, tile_h=4, block=256, ctas_per_sm=0, refill=16):
    t = gbrt_tuning()
    t.tile_w, t.tile_h, t.block, t.ctas_per_sm, t.refill = tile_w, tile_h, block, ctas_per_sm, refill
    return _check(lib.gbrt_set_tuning(ctx, C.byref(t)), "gbrt_set_tuning")


def gbrt_get_tuning(ctx):
    t = gbrt_tuning()
    _check(lib.gbrt_get_tuning(ctx, C.byref(t)), "gbrt_get_tuning")
    return dict(tile_w=t.tile_w, tile_h=t.tile_h, block=t.block, ctas_per_sm=t.ctas_per_sm, refill=t.refill)


PROFILE_ALL = 1
PROFILE_AO_WALK = 2


def gbrt_set_profiling(ctx, on=True, ao_walk_only=False):
    """Per-kernel CUDA events: off, around every kernel, or (ao_walk_only)
    only around the AO walk."""
    mode = 0 if not on else (PROFILE_AO_WALK if ao_walk_only else PROFILE_ALL)
    return _check(lib.gbrt_set_profiling(ctx, mode), "gbrt_set_profiling")


PHASES = ("primary", "ao_plan", "ao_walk", "shade")


def gbrt_phase_times(ctx):
    """Per-kernel device times (ms) of the last timed render."""
    out = (C.c_float * 4)()
    _check(lib.gbrt_phase_times(ctx, out), "gbrt_phase_times")
    return dict(zip(PHASES, [float(x) for x in out]))


def gbrt_launch_count(ctx) -> int:
    return int(lib.gbrt_launch_count(ctx))


def make_item(scene, grid, camera, width, height, ao_samples, lights, params, out_rgb, out_hit_ids=None,
              out_ao_visible=None, rows=None) -> gbrt_render_item:
    """rows=(begin, end) renders only that band of the image's rows."""
    it = gbrt_render_item()
    it.scene, it.grid = scene, grid
    if rows is not None:
        it.row_begin, it.row_end = int(rows[0]), int(rows[1])
    it.camera = camera if isinstance(camera, gbrt_camera) else make_camera(camera)
    it.width, it.height, it.ao_samples = int(width), int(height), int(ao_samples)
    it.lights = lights if isinstance(lights, gbrt_lights) else make_lights(lights)
    it.params = params if isinstance(params, gbrt_params) else make_params(params)
    rgb_b, px_b = _frame_bytes(it.camera, width, height, it.params)
    w = "make_item"
    it.out_rgb, it.out_hit_ids, it.out_ao_visible = (_buf(out_rgb, rgb_b, False, w), _buf(out_hit_ids, px_b, False, w),
                                                     _buf(out_ao_visible, px_b, False, w))
    return it


# ------------------------------------------------------------ convenience

class Renderer:
    """One context on a device + resident scenes/grids; outputs are torch tensors.

    The current torch stream is used unless ``stream`` is given.
    """

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.ctx = gbrt_create(device, self.stream)
        self._owned = []

    def upload(self, scene, lam=0.0):
        t = self.torch
        dev = f"cuda:{self.device}"
        sph = t.from_numpy(np.ascontiguousarray(scene.spheres, np.float32).reshape(-1, 4)).to(dev)
        cyl = t.from_numpy(np.ascontiguousarray(scene.cylinders, np.float32).reshape(-1, 7)).to(dev)
        col = t.from_numpy(np.ascontiguousarray(scene.color_idx, np.uint32).view(np.int32)).to(dev)
        pal = t.from_numpy(np.ascontiguousarray(scene.palette, np.float32).reshape(-1, 3)).to(dev)
        t.cuda.synchronize(self.device)
        sc = gbrt_scene_upload(self.ctx, sph, cyl, col, pal, DEVICE_PTRS)
        gr = gbrt_grid_build(self.ctx, sc, lam)
        self._owned.append((sc, gr))
        return sc, gr

    def render(self, scene, grid, camera, width, height, lights, params, ao_samples=None, ids=False, vis=False):
        t = self.torch
        dev = f"cuda:{self.device}"
        dtype = t.float64 if params.precision == FP64 else t.float32
        rgb = t.empty((height, width, 3), dtype=dtype, device=dev)
        # hit ids and AO counts: one per sub-sample, in the m-times finer raster
        m = max(1, int(getattr(camera, "aa", 1) or 1))
        hid = t.empty((m * height, m * width), dtype=t.int32, device=dev) if ids else None
        av = t.empty((m * height, m * width), dtype=t.int32, device=dev) if vis else None
        spp = params.ao_samples if ao_samples is None else ao_samples
        gbrt_render(self.ctx, scene, grid, camera, width, height, spp, lights, params, rgb, hid, av)
        return rgb, hid, av

    def free(self, scene, grid):
        gbrt_grid_free(self.ctx, grid)
        gbrt_scene_free(self.ctx, scene)
        self._owned = [(s, g) for (s, g) in self._owned if s != scene]

    def close(self):
        if self.ctx:
            for sc, gr in self._owned:
                gbrt_grid_free(self.ctx, gr)
                gbrt_scene_free(self.ctx, sc)
            self._owned = []
            gbrt_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
