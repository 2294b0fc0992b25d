"""Several views per call (the 8 mixed-resolution views of the object scene):
render_forward / render_backward launch each stage once over all views' work
items - (view, Gaussian) for the projection, (view, super-tile) for the sort,
(view, tile) for the composites - instead of once per view.

Checked here: the batched call gives the same images, loss and parameter
gradients as one call per view (the per-tile work is the same, so images are
bit-identical), calls with more views than one batch holds are split
correctly, and every view's composite matches the oracle on identical FP32
records."""
import functools

import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from helpers import cuda, workload

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def _scene_images(M):
    """Oracle fusion of all 8 frames, then each view's ray-cast (FP64 -> f32)."""
    w = workload("multiview", M=M)
    vol = oracle.Volume(w.tsdf)
    for f in w.frames:
        oracle.fuse(vol, f.depth, f.rgb, f.cam)
    out = []
    for f in w.frames:
        Ct, Dt, _, _ = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
        out.append((Ct.astype(np.float32), Dt.astype(np.float32)))
    return w, out


def _views(w, imgs, idx):
    vs = []
    for k in idx:
        f = w.frames[k]
        Ct, Dt = imgs[k]
        H, W = f.cam.height, f.cam.width
        vs.append(gps.View(f.cam, cuda(Ct), cuda(Dt), cuda(f.rgb), cuda(f.depth),
                           out_rgb=torch.empty(3, H, W, device="cuda"),
                           out_depth=torch.empty(H, W, device="cuda"),
                           out_weight=torch.empty(H, W, device="cuda")))
    return vs


@pytest.mark.parametrize("n_views", [8, 11])
@pytest.mark.parametrize("mode", [gps.BLEND_OIT, gps.BLEND_ALPHA])
def test_batched_views_equal_per_view_calls(n_views, mode):
    w, imgs = _scene_images(20000)
    idx = [k % 8 for k in range(n_views)]  # 11 views: one full batch of 8, then 3
    # the 1280 x 720 views put a Gaussian into ~25 super-tiles on average
    s = gps.settings(eps_depth=w.eps_depth, lambda_depth=1.0, blend_mode=mode, tile=(16, 8),
                     deterministic=True, pair_capacity=64 * 20000)
    g = gps.Gaussians.from_numpy(w.gaussians)
    cams = [w.frames[k].cam for k in idx]
    # batched
    vb = _views(w, imgs, idx)
    rb = gps.Renderer(g.M, cams, s)
    loss_b = torch.zeros(1, device="cuda")
    rb.forward(g, vb, loss_b)
    grads_b = g.zeros_like()
    rb.backward(g, vb, grads_b)
    # one call per view, gradients accumulated in view order
    grads_s = g.zeros_like()
    losses = []
    vs = _views(w, imgs, idx)
    for k, v in enumerate(vs):
        r = gps.Renderer(g.M, [cams[k]], s)
        lk = torch.zeros(1, device="cuda")
        r.forward(g, [v], lk)
        r.backward(g, [v], grads_s)
        losses.append(lk)
        assert r.status() == gps.GPS_OK
    torch.cuda.synchronize()
    assert rb.status() == gps.GPS_OK
    for a, b in zip(vb, vs):
        np.testing.assert_array_equal(a.out_rgb.cpu().numpy(), b.out_rgb.cpu().numpy())
        np.testing.assert_array_equal(a.out_depth.cpu().numpy(), b.out_depth.cpu().numpy())
        np.testing.assert_array_equal(a.out_weight.cpu().numpy(), b.out_weight.cpu().numpy())
    ref_loss = np.float32(0)
    for lk in losses:
        ref_loss = np.float32(ref_loss + lk.item())
    np.testing.assert_allclose(loss_b.item(), ref_loss, rtol=1e-6)
    for a, b in zip(grads_b.tensors(), grads_s.tensors()):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        scale = np.abs(b).max()
        assert scale > 0
        # same per-view terms summed in the same view order; only FMA contraction may differ
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * scale)


@pytest.mark.parametrize("mode", [gps.BLEND_OIT, gps.BLEND_ALPHA])
def test_batched_views_staged_vs_oracle(mode):
    """Oracle FP32 records written into every view's workspace; one batched
    binning + composite; each view's images against the oracle's composite."""
    w, imgs = _scene_images(4000)
    idx = list(range(8))
    s = gps.settings(eps_depth=w.eps_depth, blend_mode=mode, tile=(16, 8),
                     stages=gps.STAGE_BIN | gps.STAGE_COMPOSITE, pair_capacity=64 * 4000)
    g = gps.Gaussians.from_numpy(w.gaussians)
    cams = [w.frames[k].cam for k in idx]
    r = gps.Renderer(g.M, cams, s)
    g64 = w.gaussians.astype(np.float64)
    refs = []
    for k in idx:
        rec_o, _ = oracle.project(g64, cams[k])
        r.region(k, "records", torch.float32, r.M * 16).copy_(
            torch.from_numpy(oracle.records_f32(rec_o).reshape(-1)).cuda())
        refs.append(oracle.rounded(rec_o))
    vs = _views(w, imgs, idx)
    r.forward(g, vs)
    torch.cuda.synchronize()
    assert r.status() == gps.GPS_OK
    for k, v in zip(idx, vs):
        Ct, Dt = imgs[k]
        out = oracle.composite(refs[k], Ct, Dt, w.eps_depth, mode, f32=True)
        ok = out["amb"] == 0
        assert ok.mean() > 0.999, k
        np.testing.assert_allclose(v.out_rgb.cpu().numpy()[:, ok], out["C"][:, ok], atol=1e-5)
        np.testing.assert_allclose(v.out_depth.cpu().numpy()[ok], out["D"][ok], rtol=1e-5)
        np.testing.assert_allclose(v.out_weight.cpu().numpy()[ok], out["W"][ok], rtol=1e-5,
                                   atol=1e-6)
