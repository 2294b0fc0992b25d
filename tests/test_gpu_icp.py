"""Point-to-plane ICP tracking (Sec. 3.2, Eq. 5) on the GPU against the FP64
oracle on the same inputs (a rendered depth frame, the exact reference vertex
map): per-iteration inlier counts and residuals, the final pose, and the
known true pose.  Association decisions are taken in float32 on the GPU and
in float64 by the oracle, so a handful of pixels near a threshold may count
on one side only."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import paper_2509_11574_b300 as gps
from oracle import icp
from test_oracle_icp import tracking_case

pytestmark = pytest.mark.gpu


def _gpu_track(cam, depth, ref_V, ref_ok, T_ref, s=None):
    tr = gps.Tracker(cam, s)
    ref_cam = gps.PoseCam(cam, T_ref[:3, :3], T_ref[:3, 3])
    tr.track(torch.as_tensor(depth, dtype=torch.float32).cuda(),
             torch.as_tensor(ref_V, dtype=torch.float32).contiguous().cuda(),
             torch.as_tensor(ref_ok, dtype=torch.float32).cuda(), ref_cam)
    torch.cuda.synchronize()
    res = tr.result()
    T = icp.pose_matrix(res.R.numpy(), res.t.numpy())
    return T, tr.stats.cpu().numpy()


def _rot_err(A, B):
    return np.linalg.norm(Rotation.from_matrix(A[:3, :3] @ B[:3, :3].T).as_rotvec())


@pytest.mark.parametrize("W,H,seed", [(160, 120, 0), (160, 120, 1), (320, 240, 2), (640, 480, 0)])
def test_icp_matches_oracle_and_truth(W, H, seed):
    cam, depth, ref_V, ref_ok, T_ref, T_true = tracking_case(W, H, seed)
    K = (cam.fx, cam.fy, cam.cx, cam.cy)
    # the oracle sees the same float32 inputs the GPU does
    ref_V = ref_V.astype(np.float32)
    T_ref = T_ref.astype(np.float32).astype(np.float64)
    T_o, hist = icp.track(depth, K, ref_V.astype(np.float64), ref_ok, T_ref, T_ref)
    T_g, stats = _gpu_track(cam, depth, ref_V, ref_ok, T_ref)
    n_o = np.array([h[1] for h in hist], np.float64)
    r_o = np.array([h[2] for h in hist], np.float64)
    assert stats.shape[0] == len(hist)
    # inliers: equal up to near-threshold pixels
    np.testing.assert_allclose(stats[:, 0], n_o, rtol=2e-3, atol=3)
    # first iteration: the same pose on both sides, so the same residuals
    assert abs(stats[0, 1] - r_o[0]) <= 1e-3 * r_o[0]
    assert np.linalg.norm(T_g[:3, 3] - T_o[:3, 3]) < 5e-5
    assert _rot_err(T_g, T_o) < np.radians(2e-3)
    assert np.linalg.norm(T_g[:3, 3] - T_true[:3, 3]) < 5e-4
    assert _rot_err(T_g, T_true) < np.radians(0.02)


def test_icp_single_plane_keeps_the_pose():
    H, W, f = 24, 32, 40.0

    class Cam:
        fx = fy = f
        cx, cy = W / 2, H / 2
        width, height = W, H
    d = np.full((H, W), 2.0, np.float32)
    V = icp.vertex_map(d.astype(np.float64), (f, f, W / 2, H / 2))
    T0 = np.eye(4)
    T_g, stats = _gpu_track(Cam, d, V, d > 0, T0, gps.icp_settings(iters=(2, 1, 1)))
    np.testing.assert_array_equal(T_g, T0)
    assert stats[-1, 0] > 0
