"""Voxel-hashed TSDF (Sec. 3.2.1, as in InfiniTAM) on the GPU against the
oracle's hashing semantics: the allocated bricks, the fused values in them,
and the ray-cast; plus the ray-cast through the table against the dense
ray-cast of the same values, and the capacity error."""
import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from datagen import workloads
from helpers import cuda, workload

pytestmark = pytest.mark.gpu


def _room(n_frames=3):
    return workloads.room(n_frames=n_frames, M=16, width=160, height=120, n_vox=128)


def _fuse_both(w, n_frames, capacity=20000):
    vol_o = oracle.Volume(w.tsdf, hashed=True)
    vol_h = gps.HashTsdf(w.tsdf, capacity)
    for f in w.frames[:n_frames]:
        oracle.fuse(vol_o, f.depth, f.rgb, f.cam)
        gps.fuse_frame_hashed(vol_h, cuda(f.depth), cuda(f.rgb), f.cam)
    torch.cuda.synchronize()
    return vol_o, vol_h


def _dense_copy(w, vol_h):
    d = gps.Tsdf(w.tsdf)
    vol_h.to_dense(d)
    torch.cuda.synchronize()
    return d


@pytest.mark.parametrize("name,n_frames", [("small", 1), ("room", 3)])
def test_hashed_fusion_matches_oracle(name, n_frames):
    w = workload("small") if name == "small" else _room()
    vol_o, vol_h = _fuse_both(w, n_frames)
    assert vol_h.error() == 0
    s = w.tsdf
    nb = (s.nz // 8, s.ny // 8, s.nx // 8)
    got = np.zeros(nb, np.uint8).reshape(-1)
    bricks = vol_h.bricks().cpu().numpy()
    assert len(np.unique(bricks)) == len(bricks)          # each brick stored once
    got[bricks] = 1
    got = got.reshape(nb)
    # bricks whose band decision is within rounding of its threshold may go
    # either way; everywhere else the allocated sets are identical
    amb_b = (vol_o.amb & 2).reshape(nb[0], 8, nb[1], 8, nb[2], 8).max(axis=(1, 3, 5)) > 0
    assert amb_b.mean() < 0.1
    np.testing.assert_array_equal(got[~amb_b], vol_o.alloc[~amb_b])
    assert vol_o.alloc.sum() > 20
    # values: the dense fusion test's tolerances, on voxels of bricks both
    # sides allocated and with no near-threshold decision
    d = _dense_copy(w, vol_h)
    sdf, wt, rgbw = (t.cpu().numpy() for t in d.linear())
    both = np.repeat(np.repeat(np.repeat((got == 1) & (vol_o.alloc == 1) & ~amb_b, 8, 0), 8, 1),
                     8, 2)
    ok = both & (vol_o.amb == 0)
    assert ok.sum() > 10000
    np.testing.assert_array_equal(wt[ok], vol_o.w[ok])
    # f = eta / mu with eta = D - z_c: the kernel's z_c comes from a float
    # transform of metre-scale coordinates (within about 4e-7 m), so f is
    # within 4e-7 / mu; the running average keeps that bound, plus rounding
    tol_sdf = 2e-6 + 4e-7 / s.trunc
    np.testing.assert_allclose(sdf[ok], vol_o.sdf[ok], atol=tol_sdf)
    np.testing.assert_allclose(rgbw[..., :3][ok], vol_o.rgb[ok], atol=2e-6 * n_frames)
    np.testing.assert_array_equal(rgbw[..., 3][ok], vol_o.cw[ok])
    # bricks not stored read as unobserved
    none = np.repeat(np.repeat(np.repeat(got == 0, 8, 0), 8, 1), 8, 2)
    assert np.all(sdf[none] == 1) and np.all(wt[none] == 0)


def test_hashed_raycast_equals_dense_raycast_of_the_same_values():
    w = _room()
    _, vol_h = _fuse_both(w, 3)
    d = _dense_copy(w, vol_h)
    for f in w.frames[:3]:
        c1, d1 = gps.raycast_sdf_hashed(vol_h, f.cam)
        c2, d2 = gps.raycast_sdf(d, f.cam)
        v1 = torch.empty(f.cam.height, f.cam.width, 3, device="cuda")
        gps.raycast_sdf_hashed(vol_h, f.cam, out_vertex=v1)
        torch.cuda.synchronize()
        assert torch.equal(d1, d2) and torch.equal(c1, c2)
        assert float((d1 > 0).float().mean()) > 0.9


def test_hashed_raycast_matches_oracle():
    """Fusion and ray-cast end to end against the oracle (FP64 hashed volume):
    hit pattern, depth to 1e-4 plus the oracle's bound on an FP32 march's hit,
    and colour as in the dense ray-cast test, away from pixels whose march
    the oracle flags as near a decision.  The two volumes differ by their
    fusions' rounding and by the bricks whose allocation lies within rounding
    of its threshold (allocated on one side only), which the oracle's march
    bound does not model: a few pixels may then hit on one side only."""
    w = _room()
    vol_o, vol_h = _fuse_both(w, 3)
    f = w.frames[2]
    Ct, Dt, _, amb, derr = oracle.raycast(w.tsdf, vol_o.sdf, vol_o.rgb, f.cam, depth_err=True)
    c, d = gps.raycast_sdf_hashed(vol_h, f.cam)
    c, d = c.cpu().numpy(), d.cpu().numpy()
    ok = amb == 0
    assert ok.mean() > 0.95
    agree = (d > 0) == (Dt > 0)
    assert agree[ok].mean() > 0.999
    hit = ok & agree & (Dt > 0)
    assert np.all(np.abs(d[hit] - Dt[hit]) <= 1e-4 * Dt[hit] + derr[hit])
    assert np.abs(c[:, hit] - Ct[:, hit]).max() < 2e-3


def test_pool_overflow_is_reported():
    w = _room()
    vol_h = gps.HashTsdf(w.tsdf, capacity=40)
    f = w.frames[0]
    gps.fuse_frame_hashed(vol_h, cuda(f.depth), cuda(f.rgb), f.cam)
    torch.cuda.synchronize()
    assert vol_h.error() == gps.GPS_ERR_CAPACITY
    assert vol_h.allocated() == 40
    # the stored bricks are still usable
    c, d = gps.raycast_sdf_hashed(vol_h, f.cam)
    torch.cuda.synchronize()
    assert torch.isfinite(d).all()
