"""Pins of the oracle's TSDF fusion and ray-cast (Sec. 3.1, Sec. 3.2.1) against
closed forms: the exact truncated SDF of a plane, analytic ray/plane, ray/box and
ray/sphere intersections, and trilinear exactness on linear fields."""
import math

import numpy as np
import pytest

import oracle
from datagen import Box, Camera, Scene, Sphere, TsdfSpec, analytic_tsdf

SPEC = TsdfSpec(32, 32, 32, 0.04, (-0.64, -0.64, -0.64), 0.12, max_weight=100.0)


def axis_camera(W=40, H=30, f=35.0, cz=-1.6):
    return Camera(f, f, W / 2.0, H / 2.0, W, H, np.eye(3), np.array([0.0, 0.0, cz]))


def voxel_centres(spec):
    return spec.voxel_centres()


def test_fuse_plane_is_truncated_sdf_of_plane():
    cam = axis_camera()
    Z0 = 1.5  # plane at world z = -0.1
    depth = np.full((cam.height, cam.width), Z0)
    rgb = np.empty((3, cam.height, cam.width))
    rgb[0], rgb[1], rgb[2] = 0.25, 0.5, 0.75
    vol = oracle.Volume(SPEC)
    oracle.fuse(vol, depth, rgb, cam)
    p = voxel_centres(SPEC)
    zc = p[..., 2] - cam.t[2]
    # voxels comfortably inside the view frustum (away from the image border)
    inside = (np.abs(p[..., 0] / zc) < 0.8 * (cam.width / 2) / cam.fx) & \
             (np.abs(p[..., 1] / zc) < 0.8 * (cam.height / 2) / cam.fy) & (zc > 0.1)
    dist = Z0 - zc  # exact signed distance to the plane along its normal
    mu = SPEC.trunc
    upd = inside & (dist >= -mu)
    np.testing.assert_allclose(vol.sdf[upd], np.minimum(1.0, dist[upd] / mu), rtol=0, atol=1e-12)
    assert np.all(vol.w[upd] == 1.0)
    assert np.all(vol.w[inside & (dist < -mu)] == 0.0)
    assert np.all(vol.sdf[inside & (dist < -mu)] == 1.0)
    band = inside & (np.abs(dist) < mu)
    assert band.sum() > 100
    np.testing.assert_array_equal(vol.rgb[band], np.broadcast_to([0.25, 0.5, 0.75], vol.rgb[band].shape))
    assert np.all(vol.cw[band] == 1.0)
    assert np.all(vol.rgb[inside & (np.abs(dist) >= mu)] == 0.0)


def test_fuse_refusion_and_weight_cap():
    cam = axis_camera()
    depth = np.full((cam.height, cam.width), 1.5)
    rgb = np.full((3, cam.height, cam.width), 0.5)
    spec = TsdfSpec(32, 32, 32, 0.04, (-0.64, -0.64, -0.64), 0.12, max_weight=2.0)
    vol = oracle.Volume(spec)
    oracle.fuse(vol, depth, rgb, cam)
    sdf1 = vol.sdf.copy()
    oracle.fuse(vol, depth, rgb, cam)
    np.testing.assert_allclose(vol.sdf, sdf1, atol=1e-15)
    upd = vol.w > 0
    assert np.all(vol.w[upd] == 2.0)
    oracle.fuse(vol, depth, rgb, cam)
    assert np.all(vol.w[upd] == 2.0)  # capped at max_weight


def test_fuse_two_planes_average():
    cam = axis_camera()
    vol = oracle.Volume(SPEC)
    Za, Zb = 1.5, 1.53
    for Z in (Za, Zb):
        oracle.fuse(vol, np.full((cam.height, cam.width), Z), np.zeros((3, cam.height, cam.width)), cam)
    p = voxel_centres(SPEC)
    zc = p[..., 2] - cam.t[2]
    inside = (np.abs(p[..., 0] / zc) < 0.8 * 20 / 35) & (np.abs(p[..., 1] / zc) < 0.8 * 15 / 35)
    mu = SPEC.trunc
    both = inside & (Za - zc >= -mu)
    fa = np.minimum(1.0, (Za - zc) / mu)
    fb = np.minimum(1.0, (Zb - zc) / mu)
    np.testing.assert_allclose(vol.sdf[both], 0.5 * (fa + fb)[both], atol=1e-12)


def test_fuse_colour_nearest_pixel():
    cam = axis_camera(W=41, H=31)  # centre pixel (20, 15) lies on the optical axis
    depth = np.full((cam.height, cam.width), 1.6)
    img = np.zeros((3, cam.height, cam.width))
    img[0] = np.arange(cam.width)[None, :] / 100.0
    img[1] = np.arange(cam.height)[:, None] / 100.0
    cam.cx, cam.cy = 20.0, 15.0
    vol = oracle.Volume(SPEC)
    oracle.fuse(vol, depth, img, cam)
    # the voxel column through x = y = -0.02 (voxel centres) projects off-axis:
    p = voxel_centres(SPEC)
    zc = p[..., 2] - cam.t[2]
    u = cam.fx * p[..., 0] / zc + cam.cx
    v = cam.fy * p[..., 1] / zc + cam.cy
    band = (np.abs(1.6 - zc) < SPEC.trunc) & (np.abs(u - np.round(u)) < 0.4) & \
           (np.abs(v - np.round(v)) < 0.4) & (u > 0) & (u < 40) & (v > 0) & (v < 30)
    assert band.sum() > 20
    np.testing.assert_allclose(vol.rgb[band][:, 0], np.round(u[band]) / 100.0, atol=1e-15)
    np.testing.assert_allclose(vol.rgb[band][:, 1], np.round(v[band]) / 100.0, atol=1e-15)


def _linear_colour(p):
    return np.stack([0.5 + 0.3 * p[..., 0], 0.4 - 0.2 * p[..., 1], 0.3 + 0.25 * p[..., 2]], -1)


@pytest.mark.parametrize("tilt", [0.0, 20.0])
def test_raycast_plane_exact(tilt):
    """Trilinear interpolation and the secant step are exact on a linear SDF, so
    the hit equals the analytic ray/plane intersection to rounding."""
    th = math.radians(tilt)
    n = np.array([math.sin(th), 0.0, -math.cos(th)])  # plane normal facing the camera
    p0 = np.array([0.0, 0.0, -0.1])

    class Plane:
        def signed_distance(self, p):
            return (p - p0) @ n

    scene = Scene([Plane()], _linear_colour)
    spec = TsdfSpec(64, 64, 64, 0.02, (-0.64, -0.64, -0.64), 0.06)
    sdf, w, rgb = analytic_tsdf(scene, spec)
    cam = axis_camera(W=48, H=36, f=40.0)
    Ct, Dt, V, amb = oracle.raycast(spec, sdf, rgb, cam)
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    dc = np.stack([(ii - cam.cx) / cam.fx, (jj - cam.cy) / cam.fy, np.ones_like(ii, float)], -1)
    s = ((p0 - cam.t) @ n) / (dc @ n)  # camera depth of the analytic hit
    hitp = cam.t + dc * s[..., None]
    ok = (np.abs(hitp) < 0.55).all(-1)  # away from the volume faces
    assert ok.sum() > 500
    np.testing.assert_allclose(Dt[ok], s[ok], rtol=1e-9)
    np.testing.assert_allclose(V[ok], hitp[ok], atol=1e-9)
    np.testing.assert_allclose(Ct[:, ok].T, _linear_colour(hitp[ok]), atol=1e-9)
    # the FP32 march bounds: along a linear SDF the secant root does not move
    # with its bracket, so an FP32 march's hit depth is known to a few dozen
    # roundings (u = 2^-24) of the depth
    _, Dt2, _, amb2, err = oracle.raycast(spec, sdf, rgb, cam, depth_err=True)
    np.testing.assert_array_equal(Dt2, Dt)
    assert (amb2[ok] == 0).mean() > 0.95
    assert np.all(err[ok] <= 64 * 2.0 ** -24 * Dt[ok]) and np.all(err[ok] > 0)
    assert np.all(err[Dt == 0] == 0)
    # a volume known only to +-e per voxel: the same hits, larger bounds, and
    # with e >= 1 (any value of f possible) every pixel's march is uncertain
    _, Dt3, _, amb3, err3 = oracle.raycast(spec, sdf, rgb, cam, depth_err=True,
                                           sdf_err=np.full(sdf.shape, 1e-4))
    np.testing.assert_array_equal(Dt3, Dt)
    assert np.all(err3[ok] >= err[ok]) and np.all(amb3[amb2 != 0] != 0)
    _, _, _, amb4 = oracle.raycast(spec, sdf, rgb, cam, sdf_err=np.ones(sdf.shape))
    assert np.all(amb4[Dt > 0] != 0)


def test_raycast_box_face_and_sphere():
    box = Box(np.array([0.1, 0.05, 0.0]), np.array([0.3, 0.25, 0.2]))
    sph = Sphere(np.array([-0.05, 0.0, 0.05]), 0.35)
    spec = TsdfSpec(64, 64, 64, 0.02, (-0.64, -0.64, -0.64), 0.06)
    cam = axis_camera(W=64, H=48, f=60.0)
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    dc = np.stack([(ii - cam.cx) / cam.fx, (jj - cam.cy) / cam.fy, np.ones_like(ii, float)], -1)
    dw = dc  # identity rotation
    for prim, tol in ((box, 1e-9), (sph, 0.1 * spec.voxel)):
        scene = Scene([prim], _linear_colour)
        sdf, w, rgb = analytic_tsdf(scene, spec)
        Ct, Dt, V, amb = oracle.raycast(spec, sdf, rgb, cam)
        s = prim.hit(cam.t, dw, 1e-6)
        hit = np.isfinite(s)
        assert hit.sum() > 200
        # the discretised SDF may round silhouettes: compare the hit mask away
        # from them (pixels whose 5x5 neighbourhood agrees analytically)
        pad = np.pad(hit, 2, mode="edge")
        nb = [pad[2 + a:2 + a + hit.shape[0], 2 + b:2 + b + hit.shape[1]]
              for a in range(-2, 3) for b in range(-2, 3)]
        interior = np.all([n == hit for n in nb], axis=0)
        np.testing.assert_array_equal((Dt > 0)[interior], hit[interior])
        hit = hit & interior & (Dt > 0)
        if prim is box:
            hp = cam.t + dw * s[..., None]
            # front-face pixels at least 1.5 voxels from the face edges: linear SDF stencil
            face = hit & (np.abs(hp[..., 0] - box.c[0]) < box.h[0] - 0.03) & \
                   (np.abs(hp[..., 1] - box.c[1]) < box.h[1] - 0.03)
            assert face.sum() > 200
            np.testing.assert_allclose(Dt[face], s[face], rtol=tol)
        else:
            # sphere: trilinear of a curved SDF, hit within 0.1 voxel along the ray
            ray_len = np.linalg.norm(dw, axis=-1)
            err = np.abs(Dt[hit] - s[hit]) * ray_len[hit]
            assert err.max() < tol, err.max()


def test_raycast_misses_outside_volume():
    spec = TsdfSpec(32, 32, 32, 0.04, (-0.64, -0.64, -0.64), 0.12)
    sdf = np.ones((32, 32, 32))
    rgb = np.zeros((32, 32, 32, 3))
    cam = axis_camera()
    Ct, Dt, V, amb = oracle.raycast(spec, sdf, rgb, cam)
    assert np.all(Dt == 0) and np.all(Ct == 0)
    # camera looking away from the volume
    cam2 = Camera(35, 35, 20, 15, 40, 30, np.diag([1.0, -1.0, -1.0]), np.array([0, 0, -1.6]))
    sdf2 = np.full((32, 32, 32), -1.0)
    Ct, Dt, V, amb = oracle.raycast(spec, sdf2, rgb, cam2)
    assert np.all(Dt == 0)
