"""Gaussian insertion and removal (Sec. 3.2 "Gaussian reconstruction", App. A)
as plain numpy - TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`.

Insertion, for one frame k with second-pass outputs C*, W_G, the observed
colour C_k and the ray-cast vertex map V (world points, D_t > 0 where the ray
hit):
  1. mask: pixels that the ray-cast hit, whose colour error is above delta_c
     and whose Gaussian weight is below delta_W (Sec. 3.2).  The colour error
     is the mean over the three channels of |C* - C_k|, taken in float32 as
     (|e_r| + |e_g|) + |e_b| > 3 delta_c, so that both implementations decide
     every pixel the same way.
  2. sample: a fraction (25 %) of the mask pixels, uniformly at random; the
     draw of pixel p (row-major index) is the (p + 1)-th output of a SplitMix64
     stream seeded with `seed` (Steele, Lea and Flood, 2014), kept when its top
     24 bits are below fraction * 2^24.
  3. one new Gaussian per sampled pixel, appended in pixel order up to the
     capacity: mean V(u), colour C_k(u), opacity 0.5, a flat disc (App. A)
     whose short axis is the surface normal at u.  Disc radius s1 from the
     three mask pixels of the (2R+1)^2 window around u whose vertices are
     nearest to V(u): s1 = min(0.1, sqrt(mean squared distance)); scales
     (s1, s1, 0.1 s1).
Removal (Sec. 3.2): Gaussians with sigma < delta_sigma, or largest scale above
delta_smax or below delta_smin, are deleted; the rest keep their order.

Readings of points the paper leaves open (listed with the other readings):
- App. A writes the radius as the square root of the mean of the (unsquared)
  distances, which is not a length; the distances are read as squared, the
  initialisation of RTG-SLAM and 3DGS (root mean squared distance to the
  three nearest points).  Taken literally, neighbours one pixel apart at
  1.5 m (2.7 mm at fx = 560) would give 5 cm discs, about twenty pixel
  footprints; read as squared, the 0.1 m cap still bites where the window's
  nearest mask pixels lie across a depth discontinuity.
- Neighbours are searched among mask pixels in a (2R+1)^2 image window
  (R = 3), not among all mask pixels of the frame; fewer than three found:
  the mean over those found; none: s1 = D_t(u) / f_x (one pixel's footprint).
- The normal is the cross product of the vertex map's horizontal and vertical
  differences (central where both neighbours are hits, one-sided otherwise;
  no usable neighbour on an axis: the reversed viewing ray), turned to face
  the camera.  The disc's short axis (local z) is rotated onto its line by
  the quaternion (1 + n_z, -n_y, n_x, 0), normalised, with n's sign chosen so
  that n_z >= 0 (a disc is the same Gaussian either way).
- The removal tests are taken on the stored parameters against constants:
  logit < ln(delta_sigma / (1 - delta_sigma)), max log-scale > ln(delta_smax),
  max log-scale < ln(delta_smin), each constant rounded to float32.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, n: np.ndarray) -> np.ndarray:
    """The n-th output (n >= 1, uint64 array) of SplitMix64 seeded with `seed`:
    state_n = seed + n * gamma; z = state_n; z = (z ^ z >> 30) * C1;
    z = (z ^ z >> 27) * C2; z ^ z >> 31 (all modulo 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + n.astype(np.uint64) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def insertion_mask(C_star, W_G, C_k, D_t, delta_c=0.05, delta_w=4.0) -> np.ndarray:
    """[H][W] bool: hit, colour error above delta_c, weight below delta_w."""
    a = np.abs(np.asarray(C_star, np.float32) - np.asarray(C_k, np.float32)).astype(np.float32)
    e = (a[0] + a[1]).astype(np.float32) + a[2]
    return (np.asarray(D_t) > 0) & (e.astype(np.float32) > np.float32(3.0 * delta_c)) & \
        (np.asarray(W_G, np.float32) < np.float32(delta_w))


def sampled_pixels(mask: np.ndarray, seed: int, fraction=0.25) -> np.ndarray:
    """Row-major indices of the mask pixels the 25 % draw keeps."""
    H, W = mask.shape
    p = np.arange(H * W, dtype=np.uint64)
    z = splitmix64(seed, p + np.uint64(1))
    keep = (z >> np.uint64(40)) < np.uint64(int(fraction * (1 << 24)))
    return np.nonzero(mask.reshape(-1) & keep)[0]


def _normal(V, hit, y, x, cam_center):
    H, W = hit.shape

    def axis_diff(dy, dx):
        y0, x0, y1, x1 = y - dy, x - dx, y + dy, x + dx
        ok0 = 0 <= y0 < H and 0 <= x0 < W and hit[y0, x0]
        ok1 = 0 <= y1 < H and 0 <= x1 < W and hit[y1, x1]
        if ok0 and ok1:
            return V[y1, x1] - V[y0, x0]
        if ok1:
            return V[y1, x1] - V[y, x]
        if ok0:
            return V[y, x] - V[y0, x0]
        return None

    gx, gy = axis_diff(0, 1), axis_diff(1, 0)
    ray = V[y, x] - cam_center
    n = np.cross(gx, gy) if gx is not None and gy is not None else -ray
    nn = np.linalg.norm(n)
    if nn == 0:
        n = -ray
        nn = np.linalg.norm(n)
    n = n / nn
    if np.dot(n, ray) > 0:
        n = -n
    return n


def quat_z_to(n) -> np.ndarray:
    """Unit quaternion (w, x, y, z) rotating the local z axis onto the line of
    unit n.  A disc's covariance does not change when its short axis flips, so
    the axis is taken as the one of +-n with non-negative z: then
    w = 1 + |n_z| >= 1 and the quaternion (1 + n_z, -n_y, n_x, 0) is well
    conditioned (near n = -z it would cancel)."""
    if n[2] < 0:
        n = -np.asarray(n)
    q = np.array([1.0 + n[2], -n[1], n[0], 0.0])
    return q / np.linalg.norm(q)


def insert(V, D_t, C_star, W_G, C_k, fx, cam_center, seed, M, capacity, delta_c=0.05,
           delta_w=4.0, fraction=0.25, radius=3):
    """New Gaussians for frame k: dict of arrays (means, log_scales, quats,
    opacity_logits, rgb) in pixel order, at most capacity - M of them, plus
    the sampled pixel indices and the mask."""
    V = np.asarray(V, np.float64)
    H, W = D_t.shape
    hit = np.asarray(D_t) > 0
    mask = insertion_mask(C_star, W_G, C_k, D_t, delta_c, delta_w)
    pix = sampled_pixels(mask, seed, fraction)[:max(0, capacity - M)]
    out = {k: [] for k in ("means", "log_scales", "quats", "opacity_logits", "rgb")}
    Ck = np.asarray(C_k, np.float64)
    for p in pix:
        y, x = divmod(int(p), W)
        d2 = []
        for yy in range(max(0, y - radius), min(H, y + radius + 1)):
            for xx in range(max(0, x - radius), min(W, x + radius + 1)):
                if (yy, xx) != (y, x) and mask[yy, xx]:
                    d2.append(float(np.sum((V[yy, xx] - V[y, x]) ** 2)))
        d2.sort()
        if d2:
            s1 = min(0.1, float(np.sqrt(np.mean(d2[:3]))))
        else:
            s1 = min(0.1, float(D_t[y, x]) / fx)
        n = _normal(V, hit, y, x, np.asarray(cam_center, np.float64))
        out["means"].append(V[y, x])
        out["log_scales"].append(np.log([s1, s1, 0.1 * s1]))
        out["quats"].append(quat_z_to(n))
        out["opacity_logits"].append(0.0)
        out["rgb"].append(Ck[:, y, x])
    res = {k: np.array(v, np.float64).reshape((len(pix),) + ((3,) if k in ("means", "log_scales", "rgb") else (4,) if k == "quats" else ()))
           for k, v in out.items()}
    return res, pix, mask


def removal_keep(log_scales, opacity_logits, delta_sigma=0.005, delta_smax=0.1,
                 delta_smin=0.003) -> np.ndarray:
    """[M] bool: the Gaussians that stay (Sec. 3.2 removal criteria, read in
    logit / log-scale space against float32 constants)."""
    ls = np.asarray(log_scales, np.float32)
    lg = np.asarray(opacity_logits, np.float32)
    t_sig = np.float32(np.log(delta_sigma / (1.0 - delta_sigma)))
    t_max, t_min = np.float32(np.log(delta_smax)), np.float32(np.log(delta_smin))
    m = ls.max(axis=1)
    return ~((lg < t_sig) | (m > t_max) | (m < t_min))
