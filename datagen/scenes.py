"""Seeded synthetic RGB-D scenes, camera paths and initial Gaussian sets.

This module only manufactures inputs: analytic ray/primitive intersection for
the RGB-D frames, procedural textures, camera paths and the random initial
Gaussian parameters.  It contains none of the reconstruction method's own
arithmetic (no TSDF fusion, ray-marching, splatting or gradients), so both the
FP64 oracle and the CUDA path can consume its output without sharing code.

Conventions (shared by every consumer):
  * camera frame is OpenCV-style: x right, y down, +z forward;
  * a pose is T_wc (camera -> world): X_w = R @ X_c + t, so t is the camera
    centre in world coordinates;
  * pixel (i, j) (column i, row j) has its centre at continuous image
    coordinate (i, j), so u = fx * x / z + cx;
  * images are planar float32 arrays [C][H][W]; depth is camera z in metres,
    0 means invalid / no hit.

The stand-in workloads replace the paper's Replica, TUM-RGBD, ScanNet++ and
Azure-Kinect sequences (Sec. 4.1.2), none of which is available here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray  # (3, 3) camera -> world rotation, row-major
    t: np.ndarray  # (3,) camera centre in world coordinates

    def intrinsics(self) -> Tuple[float, float, float, float, int, int]:
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


def scaled_intrinsics(width: int, height: int) -> Tuple[float, float, float, float]:
    """fx = fy = 140 * W / 160, principal point at (W/2, H/2)."""
    f = 140.0 * width / 160.0
    return f, f, width / 2.0, height / 2.0


def look_at(eye: Sequence[float], target: Sequence[float],
            up: Sequence[float] = (0.0, -1.0, 0.0)) -> np.ndarray:
    """Camera->world rotation whose +z axis points from eye to target and whose
    -y axis is as close as possible to `up` (OpenCV: y points down)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.asarray(up, np.float64)
    # y_c points "down": -up with its component along z removed; x = y × z
    y = -up - np.dot(-up, z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    x /= np.linalg.norm(x)
    return np.stack([x, y, z], axis=1)  # columns are camera axes in world


def rotation_about(axis: Sequence[float], angle: float) -> np.ndarray:
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


# ----------------------------------------------------------------------------
# analytic scene primitives
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Sphere:
    c: np.ndarray
    r: float

    def hit(self, o, d, smin):
        oc = o - self.c
        a = np.einsum("...k,...k->...", d, d)
        b = 2.0 * np.einsum("...k,...k->...", d, oc)
        cc = np.dot(oc, oc) - self.r * self.r
        disc = b * b - 4 * a * cc
        s = np.full(a.shape, np.inf)
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        s0 = (-b - sq) / (2 * a)
        s1 = (-b + sq) / (2 * a)
        s = np.where(ok & (s0 > smin), s0, np.where(ok & (s1 > smin), s1, np.inf))
        return s

    def signed_distance(self, p):
        return np.linalg.norm(p - self.c, axis=-1) - self.r


@dataclasses.dataclass
class Box:
    c: np.ndarray
    h: np.ndarray  # half extents
    inside: bool = False  # True: a room seen from inside (hit = exit point)

    def hit(self, o, d, smin):
        tmin = np.full(d.shape[:-1], -np.inf)
        tmax = np.full(d.shape[:-1], np.inf)
        with np.errstate(divide="ignore", invalid="ignore"):
            for k in range(3):
                inv = 1.0 / d[..., k]
                t1 = (self.c[k] - self.h[k] - o[k]) * inv
                t2 = (self.c[k] + self.h[k] - o[k]) * inv
                lo = np.minimum(t1, t2)
                hi = np.maximum(t1, t2)
                np.maximum(tmin, np.where(np.isnan(lo), -np.inf, lo), out=tmin)
                np.minimum(tmax, np.where(np.isnan(hi), np.inf, hi), out=tmax)
        if self.inside:
            return np.where((tmax > smin) & (tmin <= tmax), tmax, np.inf)
        return np.where((tmin <= tmax) & (tmin > smin), tmin, np.inf)

    def signed_distance(self, p):
        q = np.abs(p - self.c) - self.h
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
        inside = np.minimum(np.max(q, axis=-1), 0.0)
        sd = outside + inside
        return -sd if self.inside else sd


@dataclasses.dataclass
class Scene:
    prims: List[object]
    colour: Callable[[np.ndarray], np.ndarray]  # (..., 3) world points -> (..., 3) rgb

    def signed_distance(self, p):
        """Union of the primitives: min of their signed distances."""
        return np.min(np.stack([pr.signed_distance(p) for pr in self.prims]), axis=0)


def render_rgbd(scene: Scene, cam: Camera, depth_noise: float = 0.0,
                rng: np.random.Generator | None = None):
    """Analytic ray casting of the primitives.

    Returns (rgb [3][H][W] f32, depth [H][W] f32, vertex [H][W][3] f64 clean world
    hit points (nan where no hit)).  Depth is camera z, optionally with additive
    N(0, depth_noise) noise on valid pixels.
    """
    H, W = cam.height, cam.width
    jj, ii = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    dc = np.stack([(ii - cam.cx) / cam.fx, (jj - cam.cy) / cam.fy, np.ones_like(ii)], -1)
    dw = dc @ cam.R.T  # world direction with camera-z component 1 per unit s
    o = cam.t.astype(np.float64)
    s = np.full((H, W), np.inf)
    for pr in scene.prims:
        s = np.minimum(s, pr.hit(o, dw, 1e-6))
    valid = np.isfinite(s)
    s_f = np.where(valid, s, 0.0)
    vertex = o + dw * s_f[..., None]
    vertex[~valid] = np.nan
    rgb = np.zeros((H, W, 3))
    if valid.any():
        rgb[valid] = scene.colour(vertex[valid])
    depth = np.where(valid, s_f, 0.0)
    if depth_noise > 0.0:
        assert rng is not None
        depth = np.where(valid, depth + rng.normal(0.0, depth_noise, size=depth.shape), 0.0)
        depth = np.where(depth > 0, depth, 0.0)
    return (np.ascontiguousarray(rgb.transpose(2, 0, 1)).astype(np.float32),
            depth.astype(np.float32), vertex)


# ----------------------------------------------------------------------------
# procedural colour
# ----------------------------------------------------------------------------
class LatticeNoise:
    """RGB ~ U[0,1] on a regular lattice, trilinearly interpolated."""

    def __init__(self, lo, hi, spacing, rng):
        self.lo = np.asarray(lo, np.float64)
        self.spacing = float(spacing)
        n = np.ceil((np.asarray(hi, np.float64) - self.lo) / spacing).astype(int) + 2
        self.vals = rng.uniform(0.0, 1.0, size=(n[0], n[1], n[2], 3))
        self.n = n

    def __call__(self, p):
        g = (p - self.lo) / self.spacing
        g = np.clip(g, 0.0, self.n - 1.000001)
        i = np.floor(g).astype(int)
        f = g - i
        out = np.zeros(p.shape[:-1] + (3,))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = ((f[..., 0] if dx else 1 - f[..., 0]) *
                         (f[..., 1] if dy else 1 - f[..., 1]) *
                         (f[..., 2] if dz else 1 - f[..., 2]))
                    out += w[..., None] * self.vals[i[..., 0] + dx, i[..., 1] + dy, i[..., 2] + dz]
        return out


class CheckerNoise:
    """10 cm 3D checker (1 / 0.5) times a 5 cm lattice value noise, in [0.2, 1]."""

    def __init__(self, lo, hi, rng, checker=0.10, spacing=0.05):
        self.noise = LatticeNoise(lo, hi, spacing, rng)
        self.checker = checker

    def __call__(self, p):
        k = np.floor(p / self.checker).astype(np.int64).sum(-1)
        chk = np.where(k % 2 == 0, 1.0, 0.5)
        return 0.2 + 0.8 * chk[..., None] * self.noise(p)


# ----------------------------------------------------------------------------
# dense TSDF geometry descriptor (storage itself is owned by the consumer)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class TsdfSpec:
    nx: int
    ny: int
    nz: int
    voxel: float
    origin: Tuple[float, float, float]
    trunc: float
    max_weight: float = 100.0

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    def voxel_centres(self) -> np.ndarray:
        """(nz, ny, nx, 3) world coordinates of voxel centres (x fastest)."""
        z, y, x = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                              indexing="ij")
        idx = np.stack([x, y, z], -1).astype(np.float64)
        return np.asarray(self.origin) + (idx + 0.5) * self.voxel


def analytic_tsdf(scene: Scene, spec: TsdfSpec):
    """Test fixture: the exact truncated signed distance of the scene sampled at
    voxel centres, clamp(dist / trunc, -1, 1), weight 1, colour from the scene's
    colour function at the voxel centre.  Linear storage, x fastest:
    returns sdf (nz, ny, nx), weight (nz, ny, nx), rgb (nz, ny, nx, 3), all f64."""
    p = spec.voxel_centres()
    dist = scene.signed_distance(p)
    sdf = np.clip(dist / spec.trunc, -1.0, 1.0)
    w = np.ones_like(sdf)
    rgb = scene.colour(p)
    return sdf, w, rgb


# ----------------------------------------------------------------------------
# Gaussian initialisation
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class GaussianSet:
    means: np.ndarray        # (M, 3)
    log_scales: np.ndarray   # (M, 3)
    quats: np.ndarray        # (M, 4) w, x, y, z (not necessarily unit)
    opacity_logits: np.ndarray  # (M,)
    rgb: np.ndarray          # (M, 3)
    sh_rest: Optional[np.ndarray] = None  # (M, (D+1)^2 - 1, 3) SH coefficients of degree 1..D

    @property
    def M(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        if self.sh_rest is None:
            return 0
        return {3: 1, 8: 2, 15: 3}[self.sh_rest.shape[1]]

    def astype(self, dt) -> "GaussianSet":
        return GaussianSet(*(None if getattr(self, f.name) is None else
                             np.ascontiguousarray(getattr(self, f.name), dtype=dt)
                             for f in dataclasses.fields(self)))

    def arrays(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logits, self.rgb]


def init_gaussians(vertex_maps: Sequence[np.ndarray], M: int, seed: int) -> GaussianSet:
    """Means on the clean surface (random valid pixels of random vertex maps) plus
    N(0, 5 mm) offsets; log-scales N(ln 1 cm, 0.3); quaternions N(0,1)^4
    normalised; opacity logits N(0, 1); colours U[0, 1]."""
    rng = np.random.default_rng(seed)
    pts = []
    for vm in vertex_maps:
        v = vm.reshape(-1, 3)
        pts.append(v[np.isfinite(v[:, 0])])
    pool_sizes = np.array([len(p) for p in pts])
    which = rng.integers(0, len(pts), size=M)
    means = np.empty((M, 3))
    for k in range(len(pts)):
        sel = np.nonzero(which == k)[0]
        if len(sel):
            means[sel] = pts[k][rng.integers(0, pool_sizes[k], size=len(sel))]
    means += rng.normal(0.0, 0.005, size=(M, 3))
    log_scales = rng.normal(math.log(0.01), 0.3, size=(M, 3))
    q = rng.normal(0.0, 1.0, size=(M, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.0, 1.0, size=M)
    rgb = rng.uniform(0.0, 1.0, size=(M, 3))
    return GaussianSet(means, log_scales, q, logits, rgb).astype(np.float32)


def with_sh(g: GaussianSet, degree: int, seed: int, scale: float = 0.1) -> GaussianSet:
    """A copy of g with SH coefficients of degree 1..`degree` drawn from
    N(0, scale^2) (float32)."""
    rng = np.random.default_rng(seed)
    K = (degree + 1) ** 2 - 1
    out = GaussianSet(*(np.array(a) for a in g.arrays()))
    out.sh_rest = rng.normal(0.0, scale, size=(g.M, K, 3)).astype(np.float32) if K else None
    return out


# ----------------------------------------------------------------------------
# scenes used by the workloads
# ----------------------------------------------------------------------------
def object_scene(seed: int = 0) -> Scene:
    """Unit-diameter sphere (r = 0.5 m) at (-0.1, 0, 0) united with an
    axis-aligned box centred at (0.35, 0.25, -0.25) with 0.2 m half-extents;
    colour = U[0,1] RGB on a 1 cm lattice (seed 0), trilinear on the surface."""
    rng = np.random.default_rng(seed)
    colour = LatticeNoise((-0.72,) * 3, (0.72,) * 3, 0.01, rng)
    return Scene([Sphere(np.array([-0.1, 0.0, 0.0]), 0.5),
                  Box(np.array([0.35, 0.25, -0.25]), np.array([0.2, 0.2, 0.2]))], colour)


def room_scene(size: float, seed: int = 2, n_objects: int = 20,
               keep_clear: Tuple[np.ndarray, float] | None = None) -> Scene:
    """A closed room of edge `size` centred at the origin with walls inset 0.1 m
    from the volume boundary, plus `n_objects` random axis-aligned boxes and
    spheres of size 0.1-0.5 m that avoid the ball `keep_clear` (camera region)."""
    rng = np.random.default_rng(seed)
    half = size / 2.0 - 0.1
    prims: List[object] = [Box(np.zeros(3), np.full(3, half), inside=True)]
    clear_c, clear_r = keep_clear if keep_clear is not None else (np.zeros(3), 0.0)
    while len(prims) < n_objects + 1:
        extent = rng.uniform(0.1, 0.5)
        c = rng.uniform(-half + extent / 2, half - extent / 2, size=3)
        if np.linalg.norm(c - clear_c) < clear_r + extent:
            continue
        if rng.uniform() < 0.5:
            prims.append(Box(c, np.full(3, extent / 2) * rng.uniform(0.6, 1.0, size=3)))
        else:
            prims.append(Sphere(c, extent / 2))
    colour = CheckerNoise((-size / 2,) * 3, (size / 2,) * 3, rng)
    return Scene(prims, colour)


def smooth_path(n_frames: int, start: np.ndarray, seed: int,
                max_step: float = 0.02, max_rot_deg: float = 1.0) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Smooth random camera path: per frame translation <= max_step and rotation
    <= max_rot_deg, velocity and angular rate low-pass filtered random walks."""
    rng = np.random.default_rng(seed)
    R = look_at(start, start + np.array([0.15, 0.05, 1.0]))
    t = start.astype(np.float64).copy()
    v = np.zeros(3)
    w = np.zeros(3)
    out = []
    for _ in range(n_frames):
        out.append((R.copy(), t.copy()))
        v = 0.8 * v + 0.2 * rng.normal(0.0, 1.0, size=3)
        w = 0.8 * w + 0.2 * rng.normal(0.0, 1.0, size=3)
        step = v / max(1.0, np.linalg.norm(v)) * max_step
        ang = math.radians(max_rot_deg) * min(1.0, np.linalg.norm(w))
        t = t + step
        if np.linalg.norm(w) > 0:
            R = rotation_about(w, ang) @ R
    return out
