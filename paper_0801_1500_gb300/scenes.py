"""Seeded synthetic inputs: protein-like molecular scenes, cameras, lights, traces.

This module only *makes inputs*. It holds none of the ray tracer's arithmetic
(no intersection, traversal, sampling or shading); the CUDA library and the
FP64 oracle each implement those on their own and both consume the arrays and
parameter values produced here.

The paper renders one VMD example scene of 26,318 objects (Sec. 2) that is not
available here; the globules below stand in for it with the same object count
and an atom/bond mix of spheres (atoms) and cylinders (bonds).

Recipe (every number below is a stated input choice, not a paper value):
  * ``n_chains = S - C`` chains; chain lengths differ by at most one sphere.
  * each chain is a random walk of 3.8 A steps starting at a uniform point of
    the ball of radius ``0.9 R``; an isotropic step that would leave the ball of
    radius ``R`` is redrawn (at most 100 draws), after which the step points to
    the ball's centre.
  * sphere radii ~ U(1.2, 2.0); cylinders of radius 0.3 join consecutive atoms
    of a chain (both bond ends are buried inside atom spheres).
  * each object takes the colour ``chain_id mod 16`` from a seeded 16-entry
    palette with channels ~ U(0.35, 1.0).
  * numpy PCG64 seeded per scene; positions are float32 values (the arrays
    both sides read are the float32 numbers).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BOND_LENGTH = 3.8
SPHERE_RADIUS_RANGE = (1.2, 2.0)
CYLINDER_RADIUS = 0.3
PALETTE_SIZE = 16


@dataclasses.dataclass
class Scene:
    """Molecular scene as plain arrays (what ``gbrt_scene_upload`` takes).

    spheres   float32 [S, 4]  centre xyz, radius
    cylinders float32 [C, 7]  end p0 xyz, end p1 xyz, radius
    color_idx uint32  [S + C] palette index per object (global id order:
                               spheres 0..S-1, then cylinders S..S+C-1)
    palette   float32 [K, 3]  linear RGB albedo
    """

    spheres: np.ndarray
    cylinders: np.ndarray
    color_idx: np.ndarray
    palette: np.ndarray
    radius: float = 0.0
    seed: int = 0

    @property
    def n_spheres(self) -> int:
        return int(self.spheres.shape[0])

    @property
    def n_cylinders(self) -> int:
        return int(self.cylinders.shape[0])

    @property
    def n_objects(self) -> int:
        return self.n_spheres + self.n_cylinders

    def nbytes(self) -> int:
        return int(self.spheres.nbytes + self.cylinders.nbytes
                   + self.color_idx.nbytes + self.palette.nbytes)

    def bounds(self):
        """Axis-aligned box of all sphere extents and cylinder end points (float64)."""
        pts = []
        if self.n_spheres:
            c = self.spheres[:, :3].astype(np.float64)
            r = self.spheres[:, 3:4].astype(np.float64)
            pts += [c - r, c + r]
        if self.n_cylinders:
            cy = self.cylinders.astype(np.float64)
            r = cy[:, 6:7]
            pts += [cy[:, 0:3] - r, cy[:, 0:3] + r, cy[:, 3:6] - r, cy[:, 3:6] + r]
        if not pts:
            return np.zeros(3), np.zeros(3)
        allp = np.concatenate(pts, axis=0)
        return allp.min(axis=0), allp.max(axis=0)


def chain_lengths(n_spheres: int, n_cylinders: int) -> List[int]:
    n_chains = n_spheres - n_cylinders
    if n_chains <= 0:
        raise ValueError("need more spheres than cylinders (one chain per S-C)")
    base, extra = divmod(n_spheres, n_chains)
    if base < 1:
        raise ValueError("chains would be empty")
    return [base + 1] * extra + [base] * (n_chains - extra)


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return v / nrm


def _random_in_ball(rng: np.random.Generator, radius: float) -> np.ndarray:
    while True:
        p = rng.uniform(-radius, radius, 3)
        if float(p @ p) <= radius * radius:
            return p


def globule(n_spheres: int, n_cylinders: int, radius: float, seed: int = 0) -> Scene:
    """Random-walk chains packed in a ball of ``radius`` (recipe in module doc)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = chain_lengths(n_spheres, n_cylinders)
    centres = np.empty((n_spheres, 3), np.float64)
    chain_of = np.empty(n_spheres, np.int64)
    cyl_pairs = []
    k = 0
    r2 = radius * radius
    for cid, length in enumerate(lengths):
        p = _random_in_ball(rng, 0.9 * radius)
        for a in range(length):
            if a > 0:
                for _ in range(100):
                    q = p + BOND_LENGTH * _unit_vectors(rng, 1)[0]
                    if float(q @ q) <= r2:
                        break
                else:
                    toward = -p / max(float(np.linalg.norm(p)), 1e-12)
                    q = p + BOND_LENGTH * toward
                cyl_pairs.append((k - 1, k))
                p = q
            centres[k] = p
            chain_of[k] = cid
            k += 1
    radii = rng.uniform(SPHERE_RADIUS_RANGE[0], SPHERE_RADIUS_RANGE[1], n_spheres)
    spheres = np.concatenate([centres, radii[:, None]], axis=1).astype(np.float32)
    c32 = spheres[:, :3]
    cyl = np.empty((len(cyl_pairs), 7), np.float32)
    cyl_chain = np.empty(len(cyl_pairs), np.int64)
    for j, (a, b) in enumerate(cyl_pairs):
        cyl[j, 0:3] = c32[a]
        cyl[j, 3:6] = c32[b]
        cyl[j, 6] = CYLINDER_RADIUS
        cyl_chain[j] = chain_of[a]
    assert cyl.shape[0] == n_cylinders
    palette = rng.uniform(0.35, 1.0, (PALETTE_SIZE, 3)).astype(np.float32)
    color_idx = np.concatenate([chain_of % PALETTE_SIZE, cyl_chain % PALETTE_SIZE]).astype(np.uint32)
    return Scene(spheres=spheres, cylinders=cyl, color_idx=color_idx, palette=palette,
                 radius=float(radius), seed=int(seed))


def make_scene(spheres, cylinders=None, color_idx=None, palette=None) -> Scene:
    """Hand-built scene from lists (tests): spheres [[x,y,z,r]], cylinders [[p0,p1,r]]."""
    sp = np.asarray(spheres if spheres is not None else np.zeros((0, 4)), np.float32).reshape(-1, 4)
    cy = np.asarray(cylinders if cylinders is not None else np.zeros((0, 7)), np.float32).reshape(-1, 7)
    n = sp.shape[0] + cy.shape[0]
    if palette is None:
        palette = np.array([[0.8, 0.7, 0.6]], np.float32)
    palette = np.asarray(palette, np.float32).reshape(-1, 3)
    if color_idx is None:
        color_idx = np.zeros(n, np.uint32)
    return Scene(spheres=sp, cylinders=cy, color_idx=np.asarray(color_idx, np.uint32),
                 palette=palette)


# --------------------------------------------------------------------------
# Camera / lights / shading parameters (plain numbers shared by both sides)
# --------------------------------------------------------------------------

CAMERA_ORTHO = 0
CAMERA_PINHOLE = 1


@dataclasses.dataclass
class Camera:
    """Orthographic (kind 0) or pinhole (kind 1) camera, all float64.

    Ortho: pixel (i, j) (column i, row j, row 0 at the top) casts the ray
      origin = eye + u*right + v*up, direction = dir, with
      u = half_w * (2 (i + 0.5) / W - 1),  v = half_h * (1 - 2 (j + 0.5) / H).
    Pinhole: origin = eye, direction = normalize(dir + u*right + v*up) with the
      same u, v (half_w, half_h are then the tangents of the half angles).
    Supersampling (aa = m > 1): each pixel casts m x m rays through the points
      (i + (a + 0.5)/m, j + (b + 0.5)/m), a, b = 0..m-1, in place of the centre
      (i + 0.5, j + 0.5), and its colour is the mean of theirs.
    """

    eye: tuple
    dir: tuple
    up: tuple
    right: tuple
    half_w: float
    half_h: float
    kind: int = CAMERA_ORTHO
    aa: int = 1


def ortho_camera(scene: Scene, width: int, height: int, angle_deg: float = 0.0,
                 margin: float = 1.05) -> Camera:
    """Orthographic view down -z of the scene, rotated by ``angle_deg`` about +y.

    The window covers the scene box (horizontal half extent = half the larger of
    the x and z extents, vertical = half the y extent) times ``margin``, widened
    on one axis to match the image aspect. The image plane sits one unit outside
    the box's bounding sphere.
    """
    lo, hi = scene.bounds()
    ctr = 0.5 * (lo + hi)
    ext = hi - lo
    hw0 = 0.5 * max(ext[0], ext[2], 1e-6) * margin
    hh0 = 0.5 * max(ext[1], 1e-6) * margin
    aspect = width / float(height)
    if hw0 / hh0 < aspect:
        hw, hh = hh0 * aspect, hh0
    else:
        hw, hh = hw0, hw0 / aspect
    th = math.radians(angle_deg)
    back = np.array([math.sin(th), 0.0, math.cos(th)])
    right = np.array([math.cos(th), 0.0, -math.sin(th)])
    dist = 0.5 * float(np.linalg.norm(ext)) + 1.0
    eye = ctr + dist * back
    return Camera(eye=tuple(float(x) for x in eye), dir=tuple(float(x) for x in -back),
                  up=(0.0, 1.0, 0.0), right=tuple(float(x) for x in right),
                  half_w=float(hw), half_h=float(hh), kind=CAMERA_ORTHO)


def pinhole_camera(scene: Scene, width: int, height: int, angle_deg: float = 0.0, fov_deg: float = 40.0,
                   margin: float = 1.05, aa: int = 1) -> Camera:
    """Pinhole view of the scene down -z, rotated by ``angle_deg`` about +y.

    The vertical field of view is ``fov_deg``; the eye sits on the view axis
    through the box centre, far enough that a ball of the box's largest half
    extent (times ``margin``) -- the globule -- fits the vertical field. ``aa``
    is the sub-pixel grid side.
    """
    lo, hi = scene.bounds()
    ctr = 0.5 * (lo + hi)
    rad = max(0.5 * float(np.max(hi - lo)), 1e-6) * margin
    hh = math.tan(math.radians(fov_deg) / 2.0)
    hw = hh * width / float(height)
    dist = rad / math.sin(math.radians(fov_deg) / 2.0)
    th = math.radians(angle_deg)
    back = np.array([math.sin(th), 0.0, math.cos(th)])
    right = np.array([math.cos(th), 0.0, -math.sin(th)])
    eye = ctr + dist * back
    return Camera(eye=tuple(float(x) for x in eye), dir=tuple(float(x) for x in -back),
                  up=(0.0, 1.0, 0.0), right=tuple(float(x) for x in right),
                  half_w=float(hw), half_h=float(hh), kind=CAMERA_PINHOLE, aa=int(aa))


def _norm(v):
    v = np.asarray(v, np.float64)
    return tuple(float(x) for x in v / np.linalg.norm(v))


@dataclasses.dataclass
class Lights:
    """Directional lights (unit vectors pointing *toward* each light)."""

    dirs: list
    intensity: list
    scale: float = 0.3      # tachyon -rescale_lights 0.3 (Sec. 2 command line)
    skylight: float = 1.0   # tachyon -add_skylight 1.0 (Sec. 2 command line)


def default_lights() -> Lights:
    return Lights(dirs=[_norm((-0.1, 0.1, 1.0)), _norm((1.0, 2.0, 0.5))],
                  intensity=[1.0, 1.0])


PRECISION_FP32 = 0   # FP32 traversal/shading; FP64 ray, hit refined in its object's frame
PRECISION_FP64 = 1   # plain FP64 throughout


@dataclasses.dataclass
class Params:
    ao_samples: int = 16
    seed: int = 0
    frame: int = 0
    precision: int = PRECISION_FP32
    eps: float = 1e-3
    ao_maxdist: float = math.inf
    k_ao: float = 0.6
    k_d: float = 0.65
    k_s: float = 0.4
    phong_exp: float = 40.0
    background: tuple = (0.0, 0.0, 0.0)
    shadows: bool = False    # direct-light shadow rays (one per light the surface faces)


# --------------------------------------------------------------------------
# The five workloads (scene sizes and frame settings)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    width: int
    height: int
    params: Params
    lights: Lights
    camera: Camera


def small_fp64(seed: int = 0) -> Workload:
    """2,000 spheres + 1,900 cylinders, radius-25 globule, 256x256, 8 spp, plain FP64."""
    sc = globule(2000, 1900, 25.0, seed)
    return Workload("small_fp64_256x256_spp8", sc, 256, 256,
                    Params(ao_samples=8, seed=seed, precision=PRECISION_FP64),
                    default_lights(), ortho_camera(sc, 256, 256))


def paper_scene(seed: int = 0) -> Scene:
    """26,318 objects: 13,500 spheres + 12,818 cylinders, radius-60 globule."""
    return globule(13500, 12818, 60.0, seed)


def paper_1mp(seed: int = 0, precision: int = PRECISION_FP32, scene: Optional[Scene] = None) -> Workload:
    sc = scene if scene is not None else paper_scene(seed)
    return Workload("paper_26318obj_965x1137_spp16", sc, 965, 1137,
                    Params(ao_samples=16, seed=seed, precision=precision),
                    default_lights(), ortho_camera(sc, 965, 1137))


def paper_17mp(seed: int = 0, precision: int = PRECISION_FP32, scene: Optional[Scene] = None) -> Workload:
    sc = scene if scene is not None else paper_scene(seed)
    return Workload("paper_26318obj_3860x4548_spp16", sc, 3860, 4548,
                    Params(ao_samples=16, seed=seed, precision=precision),
                    default_lights(), ortho_camera(sc, 3860, 4548))


ORBIT_RESOLUTIONS = [(512, 512), (965, 1137), (1920, 1080)]


def orbit_frames(scene: Scene, n_frames: int = 64, seed: int = 0):
    """360-degree orbit about +y: per frame (W, H, spp, seed=frame index, camera)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    out = []
    for k in range(n_frames):
        w, h = ORBIT_RESOLUTIONS[int(rng.integers(0, len(ORBIT_RESOLUTIONS)))]
        spp = int(rng.integers(8, 33))
        cam = ortho_camera(scene, w, h, angle_deg=360.0 * k / n_frames)
        out.append(dict(width=w, height=h, spp=spp, seed=k, frame=k, camera=cam))
    return out


def bond_pairs(n_spheres: int, n_cylinders: int) -> np.ndarray:
    """Sphere index pairs joined by the cylinders of a ``globule`` (consecutive
    atoms of each chain, in cylinder order): int64 [C, 2]."""
    pairs = []
    start = 0
    for length in chain_lengths(n_spheres, n_cylinders):
        pairs += [(start + a - 1, start + a) for a in range(1, length)]
        start += length
    return np.asarray(pairs, np.int64).reshape(-1, 2)


class MDTrajectory:
    """Molecular-dynamics-like animation of a globule, frame by frame.

    Frame k moves every atom of the base scene by a smooth bounded thermal
    displacement -- amplitude/sqrt(3) times the sum over three seeded unit
    vectors u_m of (sin(2 pi f_m k / period + phi_m) - sin(phi_m)), f_m = 1, 2,
    3 -- and turns the whole molecule by ``spin_deg`` per frame about the +y
    axis through the base box centre; bonds follow their atoms; radii and
    colours stay. Frame 0 is the base scene.
    """

    def __init__(self, scene: Scene, amplitude: float = 0.3, period: int = 64, spin_deg: float = 2.0,
                 seed: int = 0):
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        S = scene.n_spheres
        self.base = scene
        self.pairs = bond_pairs(S, scene.n_cylinders) if scene.n_cylinders else np.zeros((0, 2), np.int64)
        self.c0 = scene.spheres[:, :3].astype(np.float64)
        self.u = np.stack([_unit_vectors(rng, S) for _ in range(3)])          # [3, S, 3]
        self.phi = rng.uniform(0.0, 2.0 * math.pi, (3, S))
        self.amplitude, self.period, self.spin = float(amplitude), int(period), float(spin_deg)
        lo, hi = scene.bounds()
        self.centre = 0.5 * (lo + hi)

    def spheres(self, k: int) -> np.ndarray:
        disp = np.zeros_like(self.c0)
        for m in range(3):
            w = np.sin(2.0 * math.pi * (m + 1) * k / self.period + self.phi[m]) - np.sin(self.phi[m])
            disp += w[:, None] * self.u[m]
        c = self.c0 + (self.amplitude / math.sqrt(3.0)) * disp
        th = math.radians(self.spin * k)
        ct, st = math.cos(th), math.sin(th)
        x, z = c[:, 0] - self.centre[0], c[:, 2] - self.centre[2]
        c[:, 0] = self.centre[0] + ct * x + st * z
        c[:, 2] = self.centre[2] - st * x + ct * z
        out = self.base.spheres.copy()
        out[:, :3] = c.astype(np.float32)
        return out

    def frame(self, k: int) -> Scene:
        sp = self.spheres(k)
        cy = self.base.cylinders.copy()
        if len(self.pairs):
            cy[:, 0:3] = sp[self.pairs[:, 0], :3]
            cy[:, 3:6] = sp[self.pairs[:, 1], :3]
        return Scene(spheres=sp, cylinders=cy, color_idx=self.base.color_idx, palette=self.base.palette,
                     radius=self.base.radius, seed=self.base.seed)


SERVE_RESOLUTIONS = [(256, 256), (965, 1137), (1920, 1080), (3860, 4548)]
SERVE_SPP = [4, 16, 64]


def serving_scenes(n_scenes: int = 8, n_min: int = 1000, n_max: int = 250000, seed: int = 0,
                   chain: int = 20) -> List[Scene]:
    """Log-spaced object counts; chains of ``chain`` atoms (sphere:cylinder ~ 1:1)."""
    out = []
    for i, n in enumerate(np.geomspace(n_min, n_max, n_scenes)):
        n = int(round(n))
        n_chains = max(1, int(round(n / (2 * chain - 1))))
        s = n_chains * chain
        c = s - n_chains
        r = 60.0 * (s / 13500.0) ** (1.0 / 3.0)
        out.append(globule(s, c, r, seed + 17 * i + 1))
    return out


def poisson_trace(n_requests: int, rate_hz: float, n_scenes: int, seed: int = 0,
                  resolutions=None, spp_choices=None):
    """Seeded Poisson arrival trace of render requests."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    resolutions = resolutions or SERVE_RESOLUTIONS
    spp_choices = spp_choices or SERVE_SPP
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        reqs.append(dict(id=i, arrival_s=t, scene=int(rng.integers(0, n_scenes)), width=w, height=h,
                         spp=int(spp_choices[int(rng.integers(0, len(spp_choices)))]),
                         seed=i, angle_deg=float(rng.uniform(0.0, 360.0))))
    return reqs
