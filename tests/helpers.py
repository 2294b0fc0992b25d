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
                       exclude=None, label="", allow=None, quantile=None):
    """Per tensor, over the rows not in `exclude` and after removing the
    per-element `allow` slack: ||g - o||_inf <= norm_tol ||o||_inf, and
    elementwise |g - o| <= elem_tol |o| where |o| > 1e-3 ||o||_inf.  With
    quantile = (q, tol_all), only the fraction q of those elements must meet
    elem_tol and all of them must meet tol_all.  Returns the worst errors."""
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
        slack = np.asarray(allow[k], np.float64).reshape(o.shape) if allow is not None else 0.0
        excess = np.maximum(np.abs(g - o) - slack, 0.0)
        nerr = excess[keep].max() / scale if keep.any() else 0.0
        big = (np.abs(o) > 1e-3 * scale) & keep
        rel = excess[big] / np.abs(o)[big] if big.any() else np.zeros(1)
        eerr = rel.max()
        assert nerr <= norm_tol, (label, k, nerr)
        if quantile is None:
            assert eerr <= elem_tol, (label, k, eerr)
            worst[k] = (float(nerr), float(eerr))
        else:
            q, tol_all = quantile
            frac = float((rel <= elem_tol).mean())
            assert frac >= q, (label, k, frac)
            assert eerr <= tol_all, (label, k, eerr)
            worst[k] = (float(nerr), float(eerr), frac)
    return worst


def sign_flip_allowance(g64, cam, rec, Ct, Dt, eps, mode, ambC, ambD, nv, lam):
    """Bound on how far the parameter gradients move when the L1 residual
    signs at the flagged pixels flip: sum over those pixels of twice the
    absolute contribution of each pixel, from the oracle's own adjoint.
    Pixels are processed in batches in which no Gaussian sees two pixels, so
    the per-batch sums hold a single pixel's contribution per Gaussian."""
    import oracle
    ext = float(np.max(np.where(rec[:, oracle.R_VIS] > 0,
                                np.maximum(rec[:, oracle.R_EX], rec[:, oracle.R_EY]), 0.0)))
    sep = 2.0 * (ext + 2.0)
    M = rec.shape[0]
    total = None
    items = [("C", c, y, x) for c, y, x in zip(*np.nonzero(ambC))] + \
            [("D", 0, y, x) for y, x in zip(*np.nonzero(ambD))]
    batches = []
    for it in items:
        for b in batches:
            if all(max(abs(it[2] - o[2]), abs(it[3] - o[3])) > sep for o in b):
                b.append(it)
                break
        else:
            batches.append([it])
    for b in batches:
        dC = np.zeros_like(Ct, dtype=np.float64)
        dD = np.zeros_like(Dt, dtype=np.float64)
        for kind, c, y, x in b:
            if kind == "C":
                dC[c, y, x] = 1.0 / (3 * nv)
            else:
                dD[y, x] = lam / nv
        g2 = oracle.composite_backward(rec, Ct, Dt, eps, dC, dD, mode)
        gr = oracle.project_backward(g64, cam, g2)
        part = {k: 2.0 * np.abs(v) for k, v in gr.items()}
        total = part if total is None else {k: total[k] + part[k] for k in total}
    if total is None:
        keys = ["means", "log_scales", "quats", "opacity_logits", "rgb"]
        if getattr(g64, "sh_rest", None) is not None:
            keys.append("sh_rest")
        total = {k: 0.0 for k in keys}
    return total
