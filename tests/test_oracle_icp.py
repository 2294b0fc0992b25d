"""Pins of the ICP tracking oracle (oracle/icp.py): the SE(3) exponential
against scipy's matrix exponential, the residual Jacobian against finite
differences, the pyramid and normal maps against closed forms, and tracking
against the known pose of a rendered frame."""
import functools

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from datagen import workloads
from datagen.scenes import Camera, render_rgbd
from oracle import icp


def test_se3_exp_matches_matrix_exponential():
    rng = np.random.default_rng(0)
    for scale in (1e-9, 1e-3, 0.3, 2.0):
        xi = rng.normal(size=6) * scale
        X = np.zeros((4, 4))
        X[:3, :3] = icp.skew(xi[3:])
        X[:3, 3] = xi[:3]
        np.testing.assert_allclose(icp.se3_exp(xi), expm(X), atol=1e-12)


def test_residual_jacobian_matches_finite_differences():
    rng = np.random.default_rng(1)
    T = icp.pose_matrix(Rotation.random(random_state=rng).as_matrix(), rng.normal(size=3))
    V = rng.normal(size=(20, 3)) + [0, 0, 2]
    q = rng.normal(size=(20, 3))
    n = rng.normal(size=(20, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    P = V @ T[:3, :3].T + T[:3, 3]
    _, _, r0 = icp.normal_equations(P, q, n)
    J = np.concatenate([n, np.cross(P, n)], 1)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        rs = []
        for s in (1, -1):
            Tp = icp.se3_exp(s * e) @ T
            rs.append(icp.normal_equations(V @ Tp[:3, :3].T + Tp[:3, 3], q, n)[2])
        np.testing.assert_allclose((rs[0] - rs[1]) / (2 * h), J[:, k], atol=1e-8)
    A, b, r = icp.normal_equations(P, q, n)
    np.testing.assert_allclose(A, J.T @ J)
    np.testing.assert_allclose(b, J.T @ r0)


def test_pyramid_by_hand():
    d = np.array([[1.0, 3.0, 0.0, 0.0],
                  [5.0, 0.0, 0.0, 2.0]])
    (d0, K0), (d1, K1) = icp.pyramid(d, (100.0, 80.0, 2.0, 1.0), levels=2)
    np.testing.assert_array_equal(d1, [[3.0, 2.0]])
    assert K1 == (50.0, 40.0, 1.0, 0.5)
    # a point seen at fine coordinate u sits at u / 2 one level up, so coarse
    # pixel centres back-project through fine pixel centres
    X = np.array([0.3, -0.2, 2.0])
    u0 = K0[0] * X[0] / X[2] + K0[2]
    u1 = K1[0] * X[0] / X[2] + K1[2]
    assert abs(u1 - u0 / 2) < 1e-12


def test_normals_of_a_tilted_plane():
    H, W, f = 30, 40, 50.0
    K = (f, f, W / 2, H / 2)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    rx, ry = (xs - K[2]) / f, (ys - K[3]) / f
    z = 2.0 / (1.0 - 0.4 * rx + 0.2 * ry)          # plane z = 2 + 0.4 x - 0.2 y
    V = icp.vertex_map(z, K)
    N, ok = icp.normal_map(V, z > 0, np.zeros(3))
    want = np.array([0.4, -0.2, -1.0]) / np.linalg.norm([0.4, -0.2, -1.0])
    assert ok.sum() == (H - 2) * (W - 2)
    np.testing.assert_allclose(N[ok], np.broadcast_to(want, (ok.sum(), 3)), atol=1e-12)


def test_single_plane_leaves_the_pose_unchanged():
    # one plane constrains three of the six degrees of freedom: A is singular
    H, W, f = 24, 32, 40.0
    K = (f, f, W / 2, H / 2)
    d = np.full((H, W), 2.0)
    V = icp.vertex_map(d, K)
    T0 = np.eye(4)
    T, hist = icp.track(d, K, V, d > 0, T0, T0, iters=(2, 1, 1))
    np.testing.assert_array_equal(T, T0)
    assert hist[-1][1] > 0


@functools.lru_cache(maxsize=None)
def _frames(W, H):
    w = workloads.room(n_frames=1, M=16, width=W, height=H)
    return w


def tracking_case(W, H, seed=0):
    """Reference: the exact vertex map of the room at a frame's pose; current:
    the noise-free depth at a pose 2 cm / 1.5 degrees away."""
    w = _frames(W, H)
    f0 = w.frames[0]
    cam = f0.cam
    T_ref = icp.pose_matrix(cam.R, cam.t)
    rng = np.random.default_rng(seed)
    axis = rng.normal(size=3)
    dR = Rotation.from_rotvec(np.radians(1.5) * axis / np.linalg.norm(axis)).as_matrix()
    dt = rng.normal(size=3)
    T_true = T_ref.copy()
    T_true[:3, :3] = dR @ T_ref[:3, :3]
    T_true[:3, 3] += 0.02 * dt / np.linalg.norm(dt)
    cam1 = Camera(cam.fx, cam.fy, cam.cx, cam.cy, W, H, T_true[:3, :3], T_true[:3, 3])
    _, depth, _ = render_rgbd(w.scene, cam1, 0.0, np.random.default_rng(0))
    ref_V = np.nan_to_num(f0.vertex, nan=0.0)
    ref_ok = np.isfinite(f0.vertex[..., 0])
    return cam, depth, ref_V, ref_ok, T_ref, T_true


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tracking_recovers_a_known_pose(seed):
    cam, depth, ref_V, ref_ok, T_ref, T_true = tracking_case(160, 120, seed)
    T, hist = icp.track(depth, (cam.fx, cam.fy, cam.cx, cam.cy), ref_V, ref_ok, T_ref, T_ref)
    et = np.linalg.norm(T[:3, 3] - T_true[:3, 3])
    eR = np.linalg.norm(Rotation.from_matrix(T[:3, :3] @ T_true[:3, :3].T).as_rotvec())
    assert et < 5e-4 and eR < np.radians(0.02), (et, np.degrees(eR))
    # the residual falls from the coarse start to the end
    assert hist[-1][2] / hist[-1][1] < 0.05 * hist[0][2] / hist[0][1]
