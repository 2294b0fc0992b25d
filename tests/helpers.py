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
    """Per tensor: ||g - o||_inf <= norm_tol ||o||_inf, and elementwise
    |g - o| <= elem_tol |o| where |o| > 1e-3 ||o||_inf (rows in `exclude` skipped
    for the elementwise test).  Returns a dict of the worst errors."""
    worst = {}
    for k in keys or ref.keys():
        o = np.asarray(ref[k], np.float64)
        g = np.asarray(got[k], np.float64).reshape(o.shape)
        scale = np.abs(o).max()
        if scale == 0:
            assert np.abs(g).max() == 0, (label, k)
            continue
        nerr = np.abs(g - o).max() / scale
        big = np.abs(o) > 1e-3 * scale
        if exclude is not None:
            big &= ~exclude.reshape((-1,) + (1,) * (o.ndim - 1))
        eerr = (np.abs(g - o)[big] / np.abs(o)[big]).max() if big.any() else 0.0
        worst[k] = (float(nerr), float(eerr))
        assert nerr <= norm_tol, (label, k, nerr)
        assert eerr <= elem_tol, (label, k, eerr)
    return worst
