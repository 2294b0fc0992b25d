"""The five synthetic workloads (seeded), as plain data.

  small    : 160x120 single frame of the sphere+box scene, 64^3 x 2 cm TSDF
             (trunc 6 cm), 2,000 Gaussians, one iteration.
  room     : 30 frames at 640x480 (fx = fy = 560) along a smooth path inside a
             2.56 m room with 20 random boxes/spheres, 256^3 x 1 cm TSDF
             (trunc 3 cm), 100,000 Gaussians, 10 iterations per frame.
  grad     : one 320x240 view of the sphere+box scene, 20,000 Gaussians,
             colour + depth L1 (lambda_depth = 1), 500 finite-difference probes.
  multiview: 8 views of the sphere+box scene on a +-30 deg arc at 1.6 m with
             resolutions 320x240 / 640x480 / 1280x720, 300,000 Gaussians.
  large    : 60 frames at 1280x720 (fx = 1120) in a 5.12 m room,
             512^3 x 1 cm TSDF, 1,000,000 Gaussians.

Every array here is input data; nothing in this module runs the method.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from .scenes import (Camera, GaussianSet, TsdfSpec, init_gaussians, look_at, object_scene,
                     render_rgbd, room_scene, scaled_intrinsics, smooth_path)


@dataclasses.dataclass
class Frame:
    cam: Camera
    rgb: np.ndarray      # [3][H][W] f32
    depth: np.ndarray    # [H][W] f32 (noisy)
    vertex: np.ndarray   # [H][W][3] f64 clean world hit points (nan = no hit)


@dataclasses.dataclass
class Workload:
    name: str
    tsdf: TsdfSpec
    frames: List[Frame]
    gaussians: GaussianSet
    iters_per_frame: int
    eps_depth: float = 0.01
    lambda_depth: float = 0.0
    near: float = 0.2
    scene: Optional[object] = None


def _frames(scene, cams, noise, seed) -> List[Frame]:
    rng = np.random.default_rng(seed)
    out = []
    for cam in cams:
        rgb, depth, vertex = render_rgbd(scene, cam, noise, rng)
        out.append(Frame(cam, rgb, depth, vertex))
    return out


def object_camera(width: int, height: int, angle_deg: float = 0.0, dist: float = 1.6) -> Camera:
    fx, fy, cx, cy = scaled_intrinsics(width, height)
    a = math.radians(angle_deg)
    eye = np.array([dist * math.sin(a), 0.0, -dist * math.cos(a)])
    R = look_at(eye, np.zeros(3)) if angle_deg != 0.0 else np.eye(3)
    return Camera(fx, fy, cx, cy, width, height, R, eye)


def small(M: int = 2000, width: int = 160, height: int = 120) -> Workload:
    scene = object_scene(seed=0)
    cam = object_camera(width, height)
    frames = _frames(scene, [cam], 0.002, seed=1)
    g = init_gaussians([f.vertex for f in frames], M, seed=0)
    spec = TsdfSpec(64, 64, 64, 0.02, (-0.64, -0.64, -0.64), 0.06)
    return Workload("small", spec, frames, g, iters_per_frame=1, scene=scene)


def grad(M: int = 20000, width: int = 320, height: int = 240) -> Workload:
    w = small(M=M, width=width, height=height)
    w.name = "grad"
    w.lambda_depth = 1.0
    w.gaussians = init_gaussians([f.vertex for f in w.frames], M, seed=4)
    return w


def multiview(M: int = 300000) -> Workload:
    scene = object_scene(seed=0)
    res = [(320, 240), (640, 480), (1280, 720), (320, 240), (640, 480), (1280, 720),
           (640, 480), (320, 240)]
    angles = np.linspace(-30.0, 30.0, len(res))
    cams = [object_camera(wd, ht, float(a)) for (wd, ht), a in zip(res, angles)]
    frames = _frames(scene, cams, 0.002, seed=1)
    g = init_gaussians([f.vertex for f in frames], M, seed=0)
    spec = TsdfSpec(64, 64, 64, 0.02, (-0.64, -0.64, -0.64), 0.06)
    return Workload("multiview", spec, frames, g, iters_per_frame=1, scene=scene)


def room(n_frames: int = 30, M: int = 100000, width: int = 640, height: int = 480,
         size: float = 2.56, n_vox: int = 256, seed_scene: int = 2,
         seed_path: int = 3) -> Workload:
    start = np.array([0.0, 0.0, -0.35 * size / 2.56])
    scene = room_scene(size, seed=seed_scene, keep_clear=(start, 0.75))
    fx, fy, cx, cy = scaled_intrinsics(width, height)
    cams = [Camera(fx, fy, cx, cy, width, height, R, t)
            for R, t in smooth_path(n_frames, start, seed_path)]
    frames = _frames(scene, cams, 0.002, seed=seed_path + 100)
    g = init_gaussians([f.vertex for f in frames], M, seed=0)
    spec = TsdfSpec(n_vox, n_vox, n_vox, size / n_vox, (-size / 2,) * 3, 0.03)
    return Workload("room", spec, frames, g, iters_per_frame=10, scene=scene)


def large() -> Workload:
    w = room(n_frames=60, M=1000000, width=1280, height=720, size=5.12, n_vox=512)
    w.name = "large"
    return w


def tiny(M: int = 64, width: int = 40, height: int = 30) -> Workload:
    """A few-tile case for brute-force checks (ragged tiles, 32^3 TSDF)."""
    scene = object_scene(seed=0)
    cam = object_camera(width, height)
    frames = _frames(scene, [cam], 0.002, seed=1)
    g = init_gaussians([f.vertex for f in frames], M, seed=7)
    spec = TsdfSpec(32, 32, 32, 0.04, (-0.64, -0.64, -0.64), 0.12)
    return Workload("tiny", spec, frames, g, iters_per_frame=1, scene=scene)
