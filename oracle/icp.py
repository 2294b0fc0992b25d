"""Camera tracking by point-to-plane ICP (Sec. 3.2 "Camera tracking", Eq. 5,
after KinectFusion and InfiniTAM) in plain numpy, FP64 - TEST INFRASTRUCTURE
ONLY, like the rest of `oracle/`.

Given the current depth map D_k, the intrinsics K, the reference vertex map V*
and normal map N* (world frame, ray-cast at the previous pose T_ref, full
resolution) and an initial camera->world pose T, Gauss-Newton minimises

    E(T) = sum_u ((T V_k(u) - V*(u^)) . N*(u^))^2

over a depth pyramid, coarsest level first.  One iteration at one level:
  1. p = T V_k(u) for every pixel u of the level with a depth and a normal;
  2. u^ = nearest pixel of pi(K, T_ref^-1 p) (projective data association
     into the reference view, full resolution; nearest = floor(x + 0.5));
  3. u is an inlier when u^ lies in the image, V*(u^) and N*(u^) exist,
     |p - V*(u^)| < eps_d and angle(R N_k(u), N*(u^)) < eps_theta;
  4. r = (p - q) . n and J = [n^T, (p x n)^T], the derivative of r for the
     update T <- exp(xi^) T with xi = (v, w) (translation, rotation);
  5. A = sum J^T J, b = sum J^T r, xi = -A^-1 b, T <- exp(xi^) T.

Readings of points the paper leaves open (listed with the other readings):
- 3 levels; level l + 1 holds the mean of the valid depths of each 2x2 block
  of level l (0 when none is valid), with intrinsics f / 2 and c / 2, as
  InfiniTAM halves them: coarse pixel i then sits on fine pixel 2i, so a
  coarse point at the reference pose projects onto a reference pixel centre.
  (With c' = (c - 0.5) / 2, the block's own centre, it would land on a pixel
  corner, where the nearest-pixel association is a four-way tie.)
- Iterations per level, finest first, 10, 5, 4 and the rejection thresholds
  eps_d = 0.1 m, eps_theta = 20 degrees (KinectFusion's values).
- Normals (current levels and reference): cross product of the central
  differences (V(x+1) - V(x-1)) x (V(y+1) - V(y-1)), turned towards the
  camera; a pixel lacking any of its four neighbours has no normal.
- An iteration with fewer than six inliers, or whose A is not positive
  definite with every Cholesky pivot above 1e-6 of A's largest diagonal entry
  (fewer than six well-determined directions), leaves T unchanged.
"""
from __future__ import annotations

import math

import numpy as np

LEVELS = 3
ITERS = (10, 5, 4)      # finest level first
EPS_D = 0.1
EPS_THETA_DEG = 20.0


def skew(a) -> np.ndarray:
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def se3_exp(xi) -> np.ndarray:
    """4x4 exp of the twist xi = (v, w): rotation by Rodrigues' formula,
    translation V v with V = I + (1 - cos t)/t^2 [w] + (t - sin t)/t^3 [w]^2."""
    v, w = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    t = float(np.linalg.norm(w))
    W = skew(w)
    if t < 1e-12:
        R = np.eye(3) + W
        V = np.eye(3) + 0.5 * W
    else:
        R = np.eye(3) + math.sin(t) / t * W + (1 - math.cos(t)) / t ** 2 * (W @ W)
        V = np.eye(3) + (1 - math.cos(t)) / t ** 2 * W + (t - math.sin(t)) / t ** 3 * (W @ W)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ v
    return T


def pose_matrix(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = np.asarray(R, np.float64).reshape(3, 3)
    T[:3, 3] = np.asarray(t, np.float64).reshape(3)
    return T


def pyramid(depth, K, levels=LEVELS):
    """[(depth_l, (fx, fy, cx, cy)_l)] for l = 0 .. levels - 1."""
    out = [(np.asarray(depth, np.float64), tuple(float(k) for k in K))]
    for _ in range(levels - 1):
        d, (fx, fy, cx, cy) = out[-1]
        H, W = d.shape[0] // 2, d.shape[1] // 2
        b = d[:2 * H, :2 * W].reshape(H, 2, W, 2)
        n = (b > 0).sum(axis=(1, 3))
        s = np.where(b > 0, b, 0.0).sum(axis=(1, 3))
        out.append((np.where(n > 0, s / np.maximum(n, 1), 0.0),
                    (fx / 2, fy / 2, cx / 2, cy / 2)))
    return out


def vertex_map(depth, K) -> np.ndarray:
    """Camera-frame points [H][W][3] (zero where depth <= 0)."""
    fx, fy, cx, cy = K
    H, W = depth.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    z = np.where(depth > 0, depth, 0.0)
    return np.stack([(xs - cx) / fx * z, (ys - cy) / fy * z, z], -1)


def normal_map(V, valid, centre) -> tuple:
    """Unit normals [H][W][3] and their mask: central differences in x and y,
    all four neighbours valid, turned to face `centre`."""
    H, W = valid.shape
    ok = np.zeros((H, W), bool)
    ok[1:-1, 1:-1] = valid[1:-1, 1:-1] & valid[1:-1, 2:] & valid[1:-1, :-2] & \
        valid[2:, 1:-1] & valid[:-2, 1:-1]
    dx = np.zeros((H, W, 3))
    dy = np.zeros((H, W, 3))
    dx[1:-1, 1:-1] = V[1:-1, 2:] - V[1:-1, :-2]
    dy[1:-1, 1:-1] = V[2:, 1:-1] - V[:-2, 1:-1]
    n = np.cross(dx, dy)
    nn = np.linalg.norm(n, axis=-1)
    ok &= nn > 0
    n = n / np.where(nn > 0, nn, 1.0)[..., None]
    away = ((V - np.asarray(centre, np.float64)) * n).sum(-1) > 0
    N = np.where(away[..., None], -n, n)
    return np.where(ok[..., None], N, 0.0), ok


def reference_normals(ref_V, ref_valid, T_ref):
    return normal_map(ref_V, ref_valid, T_ref[:3, 3])


def associate(T, Vl, Nl, okl, ref_V, ref_N, ref_ok, T_ref, K0, eps_d=EPS_D,
              eps_theta_deg=EPS_THETA_DEG):
    """Inlier points p, reference points q, normals n (world) for pose T."""
    R, t = T[:3, :3], T[:3, 3]
    P = Vl[okl] @ R.T + t
    Nc = Nl[okl] @ R.T
    Rr, tr = T_ref[:3, :3], T_ref[:3, 3]
    X = (P - tr) @ Rr                    # reference camera frame: R_ref^T (p - t_ref)
    fx, fy, cx, cy = K0
    H, W = ref_ok.shape
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.floor(fx * X[:, 0] / X[:, 2] + cx + 0.5)
        v = np.floor(fy * X[:, 1] / X[:, 2] + cy + 0.5)
    inside = (X[:, 2] > 0) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    ui = np.where(inside, u, 0).astype(np.int64)
    vi = np.where(inside, v, 0).astype(np.int64)
    q = ref_V[vi, ui]
    n = ref_N[vi, ui]
    keep = inside & ref_ok[vi, ui]
    keep &= np.linalg.norm(P - q, axis=1) < eps_d
    keep &= (Nc * n).sum(1) > math.cos(math.radians(eps_theta_deg))
    return P[keep], q[keep], n[keep]


def normal_equations(P, q, n):
    """A = sum J^T J, b = sum J^T r with r = (p - q).n, J = [n, p x n]."""
    r = ((P - q) * n).sum(1)
    J = np.concatenate([n, np.cross(P, n)], 1)
    return J.T @ J, J.T @ r, r


def gauss_newton_step(A, b):
    """xi = -A^-1 b, or None when A is not positive definite or a Cholesky
    pivot L_jj^2 is at most 1e-6 of A's largest diagonal entry."""
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        return None
    if np.min(np.diag(L)) ** 2 <= 1e-6 * np.max(np.diag(A)):
        return None
    y = np.linalg.solve(L, -b)
    return np.linalg.solve(L.T, y)


def track(depth, K, ref_V, ref_valid, T_ref, T_init, iters=ITERS, eps_d=EPS_D,
          eps_theta_deg=EPS_THETA_DEG, levels=LEVELS):
    """Pose estimate (4x4 camera->world) and the per-iteration history
    [(level, inliers, sum r^2 before the update)]."""
    ref_V = np.asarray(ref_V, np.float64)
    ref_N, ref_ok = reference_normals(ref_V, ref_valid, T_ref)
    T = np.array(T_init, np.float64)
    hist = []
    pyr = pyramid(depth, K, levels)
    for lvl in range(levels - 1, -1, -1):
        d, Kl = pyr[lvl]
        Vl = vertex_map(d, Kl)
        Nl, okN = normal_map(Vl, d > 0, np.zeros(3))
        okl = (d > 0) & okN
        for _ in range(iters[lvl]):
            P, q, n = associate(T, Vl, Nl, okl, ref_V, ref_N, ref_ok, T_ref, K, eps_d,
                                eps_theta_deg)
            A, b, r = normal_equations(P, q, n)
            hist.append((lvl, len(r), float((r * r).sum())))
            xi = gauss_newton_step(A, b) if len(r) >= 6 else None
            if xi is not None:
                T = se3_exp(xi) @ T
    return T, hist
