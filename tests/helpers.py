"""Shared set-up of the parity tests: oracle-side inputs (fusion + ray-cast in
FP64, then rounded to float32) and the matching device-side views."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle
from datagen import workloads


@functools.lru_cache(maxsize=8)
def workload(name: str, **kw):
    return getattr(workloads, name)(**kw)


def oracle_sdf_images(w, frame: int = 0, n_fuse: int = 1):
    """Fuse the first n_fuse frames (FP64 oracle) and ray-cast `frame`.
    Returns C_t, D_t as float32 plus the oracle volume and ray-cast ambiguity."""
    vol = oracle.Volume(w.tsdf)
    for k in range(n_fuse):
        f = w.frames[k]
        oracle.fuse(vol, f.depth, f.rgb, f.cam)
    f = w.frames[frame]
    Ct, Dt, V, amb = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
    return Ct.astype(np.float32), Dt.astype(np.float32), vol, amb


def cuda(a) -> torch.Tensor:
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


def rel_err(a, b, floor):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def assert_grads_close(got: dict, ref: dict, keys=None, norm_tol=1e-4, elem_tol=1e-4,
                       exclude=None, label=""):
    """Per tensor, over the rows not in `exclude`: ||g - o||_inf <= norm_tol
    ||o||_inf, and elementwise |g - o| <= elem_tol |o| where |o| > 1e-3
    ||o||_inf.  Returns the worst errors."""
    worst = {}
    for k in keys or ref.keys():
        o = np.asarray(ref[k], np.float64)
        g = np.asarray(got[k], np.float64).reshape(o.shape)
        scale = np.abs(o).max()
        if scale == 0:
            assert np.abs(g).max() == 0, (label, k)
            continue
        keep = np.ones(o.shape, bool)
        if exclude is not None:
            keep &= ~exclude.reshape((-1,) + (1,) * (o.ndim - 1))
        err = np.abs(g - o)
        nerr = err[keep].max() / scale if keep.any() else 0.0
        big = (np.abs(o) > 1e-3 * scale) & keep
        eerr = (err[big] / np.abs(o)[big]).max() if big.any() else 0.0
        assert nerr <= norm_tol, (label, k, nerr)
        assert eerr <= elem_tol, (label, k, eerr)
        worst[k] = (float(nerr), float(eerr))
    return worst


U32 = 2.0 ** -24  # unit roundoff of binary32
# A kernel's FP32 sum of one Gaussian's per-pixel terms: a lane walks at most
# 32 pixels of its block in one FMA chain, the blocks' partials meet in
# atomics (at most about 30 per tile row of a large Gaussian), each term
# carries a few roundings plus ex2.approx (2^-22) and sigma's record error
# (2e-7): 128 u covers the sum's gamma_n and the terms' own errors.
KAPPA_SUM = 128


def record_bounds(W: int, H: int) -> dict:
    """The record errors the oracle's bands (oracle.bands_for) assume, per
    Gaussian: conic entries within 2e-6 of |a| + 2|b| + |c|, mean within
    4 u (W + H) px, qmax and sigma within 2e-7, depth within 2.3e-7 (all
    relative; the depth band adds the threshold's own rounding, 2 u)."""
    return dict(conic=2e-6, mean=4.0 * U32 * (W + H), qmax=2e-7, sigma=2e-7, depth=2.3e-7)


def record_errors(rec_g: np.ndarray, rec_o: np.ndarray, keep: np.ndarray) -> dict:
    """Worst error of the kernel's FP32 records (16 floats per Gaussian) against
    the oracle's FP64 records over the Gaussians in `keep`."""
    o = rec_o[keep]
    g = rec_g[keep].astype(np.float64)
    cn = np.abs(o[:, oracle.R_CA]) + 2 * np.abs(o[:, oracle.R_CB]) + np.abs(o[:, oracle.R_CC])
    con = np.abs(g[:, 4:7] - o[:, [oracle.R_CA, oracle.R_CB, oracle.R_CC]]).max(1) / cn
    mean = np.abs(g[:, 0:2] - o[:, [oracle.R_MX, oracle.R_MY]]).max(1)
    rel = lambda kg, ko: np.abs(g[:, kg] - o[:, ko]) / np.abs(o[:, ko])
    out = dict(conic=con, mean=mean, qmax=rel(7, oracle.R_QMAX), sigma=rel(3, oracle.R_SIG),
               depth=rel(2, oracle.R_D))
    return {k: float(v.max()) if v.size else 0.0 for k, v in out.items()}


def assert_record_bounds(rec_g, rec_o, keep, W, H, label=""):
    errs = record_errors(rec_g, rec_o, keep)
    for k, b in record_bounds(W, H).items():
        assert errs[k] <= b, (label, k, errs[k], b)
    return errs


def conic_cond(rec: np.ndarray) -> np.ndarray:
    """cond(Sigma_2D) = cond(conic), per Gaussian (1 where invisible)."""
    a, b, c = rec[:, oracle.R_CA], rec[:, oracle.R_CB], rec[:, oracle.R_CC]
    h = 0.5 * (a + c)
    disc = np.sqrt(0.25 * (a - c) ** 2 + b * b)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = (h + disc) / (h - disc)
    return np.where(np.isfinite(k) & (k > 0) & (rec[:, oracle.R_VIS] > 0), k, 1.0)


def projection_rounding(gs, cam, g2: np.ndarray, rec: np.ndarray) -> np.ndarray:
    """FP32 error bound of the projection adjoint per Gaussian and parameter
    ([M][P]), from the 2D gradient g2 it is fed:
        (8 cond(Sigma_2D) + 64) u |adjoint|_mag,
    |adjoint|_mag the oracle's adjoint evaluated in magnitude arithmetic
    (oracle.project_backward_magnitude: every term's |.| summed, so the
    cancellations of the quaternion normalisation and of dL/dSigma_2D count
    at their full size).  The chain has a few dozen roundings on its longest
    path (64 u); its inputs come from the kernel's own FP32 projection, where
    the conic, the inverse of Sigma_2D, carries about u cond(Sigma_2D) and
    enters dL/dSigma_2D = -C dL/dC C twice (8 u cond with margin)."""
    mag = params_matrix(oracle.project_backward_magnitude(gs, cam, g2), rec.shape[0])
    return (8.0 * conic_cond(rec)[:, None] + 64.0) * U32 * mag


def assert_projection_adjoint(got: dict, ref: dict, gs, cam, g2, rec, keep, label="", rel=1e-4):
    """The projection adjoint fed identical 2D gradients g2: per element,
    rel |o| + projection_rounding where |o| > 1e-3 ||o||_inf, and
    rel ||o||_inf + projection_rounding everywhere, over the Gaussians in
    `keep`.  Returns the worst ratio of error to bound per tensor."""
    M = rec.shape[0]
    slack = oracle.split_params(projection_rounding(gs, cam, np.asarray(g2, np.float64), rec), ref)
    worst = {}
    for k in ref:
        o = np.asarray(ref[k], np.float64).reshape(M, -1)[keep]
        g = np.asarray(got[k], np.float64).reshape(M, -1)[keep]
        sl = slack[k].reshape(M, -1)[keep]
        scale = np.abs(o).max()
        err = np.abs(g - o)
        big = np.abs(o) > 1e-3 * scale
        assert np.all(err <= rel * scale + sl), (label, k, ((err - sl) / scale).max())
        assert np.all(err[big] <= rel * np.abs(o[big]) + sl[big]), \
            (label, k, ((err - sl)[big] / np.abs(o[big])).max())
        worst[k] = float(np.max(err[big] / (rel * np.abs(o[big]) + sl[big])))
    return worst


def params_matrix(d: dict, M: int) -> np.ndarray:
    """dict of per-parameter arrays (PARAM_KEYS order) -> [M][P]."""
    return np.concatenate([np.asarray(d[k], np.float64).reshape(M, -1)
                           for k in oracle.PARAM_KEYS if k in d], 1)


def gaussians_over(mask: np.ndarray, rec: np.ndarray) -> np.ndarray:
    """Visible Gaussians whose candidate box (extent + 1 px, as the oracle's
    lists) contains a pixel of `mask`."""
    H, W = mask.shape
    sat = np.zeros((H + 1, W + 1), np.int64)
    sat[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.int64), 0), 1)
    vis = rec[:, oracle.R_VIS] > 0
    x0 = np.clip(np.ceil(rec[:, oracle.R_MX] - rec[:, oracle.R_EX] - 1), 0, W - 1)
    x1 = np.clip(np.floor(rec[:, oracle.R_MX] + rec[:, oracle.R_EX] + 1), 0, W - 1)
    y0 = np.clip(np.ceil(rec[:, oracle.R_MY] - rec[:, oracle.R_EY] - 1), 0, H - 1)
    y1 = np.clip(np.floor(rec[:, oracle.R_MY] + rec[:, oracle.R_EY] + 1), 0, H - 1)
    ok = vis & np.isfinite(x0 + x1 + y0 + y1) & (x0 <= x1) & (y0 <= y1)
    x0, x1, y0, y1 = (np.where(ok, v, 0).astype(np.int64) for v in (x0, x1, y0, y1))
    cnt = sat[y1 + 1, x1 + 1] - sat[y0, x1 + 1] - sat[y1 + 1, x0] + sat[y0, x0]
    return ok & (cnt > 0)


def projection_skip(rec: np.ndarray, proj_amb: np.ndarray, H: int, W: int):
    """Pixels a Gaussian whose visibility or image-border decision lies near
    its threshold may touch (its box + 2 px), and the Gaussians it leaves out:
    those over such pixels, plus those whose Jacobian clamp is near its
    threshold (their own gradient only: the clamp is continuous)."""
    skip = np.zeros((H, W), bool)
    for i in np.nonzero(proj_amb & 5)[0]:
        if rec[i, oracle.R_VIS] == 0 and proj_amb[i] & 1:
            skip[:] = True  # its footprint is unknown here: nothing can be checked
            break
        x0 = int(max(0, rec[i, oracle.R_MX] - rec[i, oracle.R_EX] - 2))
        x1 = int(min(W - 1, rec[i, oracle.R_MX] + rec[i, oracle.R_EX] + 2))
        y0 = int(max(0, rec[i, oracle.R_MY] - rec[i, oracle.R_EY] - 2))
        y1 = int(min(H - 1, rec[i, oracle.R_MY] + rec[i, oracle.R_EY] + 2))
        if x0 <= x1 and y0 <= y1:
            skip[y0:y1 + 1, x0:x1 + 1] = True
    excl = gaussians_over(skip, rec) | ((proj_amb & 5) != 0) | ((proj_amb & 2) != 0)
    return skip, excl


def envelope_slack(env: dict, JT: np.ndarray, rec: np.ndarray, gs, cam) -> np.ndarray:
    """[M][P]: what a kernel's parameter gradient may differ by from the
    oracle's beyond 1e-4 of it (see assert_grads_in_envelope)."""
    aJ = np.abs(JT)
    return (env["allow3"] + np.einsum("mpc,mc->mp", aJ, env["s2q"])
            + KAPPA_SUM * U32 * np.einsum("mpc,mc->mp", aJ, env["s2"])
            + projection_rounding(gs, cam, env["g2ref"], rec))


def assert_grads_in_envelope(got: dict, ref: dict, env: dict, JT: np.ndarray, rec: np.ndarray,
                             exclude: np.ndarray, gs, cam, label="", rel=1e-4):
    """Per parameter tensor and element, the criterion at `rel`:
        |g - o| <= rel |o| + slack            where |o| > 1e-3 ||o||_inf,
        |g - o| <= rel ||o||_inf + slack      everywhere,
    over the Gaussians not in `exclude`, with
        slack = allow3                        (decisions within the FP32 bands)
              + |J^T| s2q                     (alpha's error from q's band)
              + KAPPA_SUM u |J^T| s2          (FP32 sums of the terms)
              + projection_rounding           (the projection adjoint in FP32),
    every term from the oracle's own per-pixel terms (`oracle.envelope`).
    Returns what the check saw."""
    M = rec.shape[0]
    slack = envelope_slack(env, JT, rec, gs, cam)
    sl = oracle.split_params(slack, ref)
    al = oracle.split_params(env["allow3"], ref)
    keep = ~exclude
    stats = {"gaussians_excluded": float(exclude.mean()),
             "gaussians_with_decision_allowance": float((env["allow3"][keep].max(1) > 0).mean())}
    for k in ref:
        o = np.asarray(ref[k], np.float64).reshape(M, -1)[keep]
        g = np.asarray(got[k], np.float64).reshape(M, -1)[keep]
        s = sl[k].reshape(M, -1)[keep]
        a = al[k].reshape(M, -1)[keep]
        scale = np.abs(o).max()
        if scale == 0:
            assert np.all(np.abs(g) <= s), (label, k)
            continue
        err = np.abs(g - o)
        big = np.abs(o) > 1e-3 * scale
        assert np.all(err <= rel * scale + s), (label, k, "norm", ((err - s) / scale).max())
        assert np.all(err[big] <= rel * np.abs(o[big]) + s[big]), \
            (label, k, "elementwise", ((err - s)[big] / np.abs(o[big])).max())
        free = big & (a == 0)  # elements no ambiguous decision touches
        stats[k] = {"raw_within_rel": float(np.mean(err[big] <= rel * np.abs(o[big]))),
                    "raw_within_rel_untouched": float(np.mean(err[free] <= rel * np.abs(o[free])))
                    if free.any() else None,
                    "worst_err_over_bound": float(np.max(err[big] / (rel * np.abs(o[big]) + s[big]))),
                    "allowance_above_rel": float(np.mean(a[big] > rel * np.abs(o[big])))}
    return stats
