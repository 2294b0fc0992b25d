"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the
benchmark.  Holds no part of the reconstruction method's arithmetic."""
from .scenes import (Box, Camera, GaussianSet, Scene, Sphere, TsdfSpec, analytic_tsdf,
                     init_gaussians, look_at, object_scene, render_rgbd, room_scene,
                     rotation_about, scaled_intrinsics, smooth_path)
from . import workloads

__all__ = ["Box", "Camera", "GaussianSet", "Scene", "Sphere", "TsdfSpec", "analytic_tsdf",
           "init_gaussians", "look_at", "object_scene", "render_rgbd", "room_scene",
           "rotation_about", "scaled_intrinsics", "smooth_path", "workloads"]
