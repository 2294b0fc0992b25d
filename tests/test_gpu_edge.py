"""Degenerate and boundary cases of the render path on the GPU: no Gaussians,
every Gaussian culled, no valid pixel, an image smaller than one tile, a
Gaussian covering the whole image, and the sort-free default against the
depth-sorted order."""
import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from datagen import GaussianSet
from datagen.workloads import object_camera
from helpers import cuda, oracle_sdf_images, workload

pytestmark = pytest.mark.gpu


def _render(gs, cam, Ct, Dt, Ctgt, Dtgt, **kw):
    H, W = cam.height, cam.width
    s = gps.settings(**kw)
    r = gps.Renderer(max(gs.M, 1), [cam], s)
    g = gps.Gaussians.from_numpy(gs)
    v = gps.View(cam, cuda(Ct), cuda(Dt), cuda(Ctgt), cuda(Dtgt),
                 out_rgb=torch.empty(3, H, W, device="cuda"),
                 out_depth=torch.empty(H, W, device="cuda"),
                 out_weight=torch.empty(H, W, device="cuda"))
    loss = torch.full((1,), -1.0, device="cuda")
    r.forward(g, [v], loss)
    grads = g.zeros_like()
    r.backward(g, [v], grads)
    torch.cuda.synchronize()
    assert r.status() == gps.GPS_OK
    return (v.out_rgb.cpu().numpy(), v.out_depth.cpu().numpy(), v.out_weight.cpu().numpy(),
            loss.item(), grads)


def _empty_set(M=0):
    z = lambda *s: np.zeros(s, np.float32)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (M, 1))
    return GaussianSet(z(M, 3), z(M, 3), q, z(M), z(M, 3))


def test_no_gaussians_returns_the_sdf_image_and_its_loss():
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    c, d, wg, L, grads = _render(_empty_set(), f.cam, Ct, Dt, f.rgb, f.depth, tile=(16, 8))
    np.testing.assert_array_equal(c, Ct)          # (C_t + 0) / (1 + 0)
    np.testing.assert_array_equal(d, Dt)
    assert np.all(wg == 0)
    L_o = oracle.loss(Ct, Dt, f.rgb, f.depth, Dt)[0]
    assert abs(L - L_o) <= 1e-5 * L_o


def test_every_gaussian_culled_matches_no_gaussians():
    """Gaussians behind the near plane, outside the frustum, or too faint:
    the image is the SDF image bit for bit and every gradient is zero."""
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    rng = np.random.default_rng(0)
    M = 300
    # the camera sits at z = -1.6 looking along +z
    means = np.concatenate([rng.normal(0, 0.1, (100, 3)) + [0, 0, -2.2],      # behind the camera
                            rng.normal(0, 0.1, (100, 3)) + [40.0, 0, 1.0],    # far outside
                            rng.normal(0, 0.1, (100, 3))]).astype(np.float32)  # faint
    logits = np.concatenate([np.zeros(200), np.full(100, -7.0)]).astype(np.float32)
    gs = GaussianSet(means, np.full((M, 3), np.log(0.01), np.float32),
                     np.tile(np.array([1, 0, 0, 0], np.float32), (M, 1)), logits,
                     np.full((M, 3), 0.5, np.float32))
    c, d, wg, L, grads = _render(gs, f.cam, Ct, Dt, f.rgb, f.depth, tile=(16, 8))
    np.testing.assert_array_equal(c, Ct)
    assert np.all(wg == 0)
    assert float(grads.flat().abs().max()) == 0.0


def test_no_valid_pixel_gives_zero_loss_and_gradients():
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    c, d, wg, L, grads = _render(w.gaussians, f.cam, Ct, Dt, f.rgb, np.zeros_like(f.depth),
                                 tile=(16, 8))
    assert L == 0.0
    assert float(grads.flat().abs().max()) == 0.0
    assert wg.max() > 0                           # the blend itself still ran


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (8, 8), (32, 8)])
def test_image_smaller_than_a_tile_matches_oracle(tile):
    """13 x 7 pixels (one partial tile) with Gaussians around the view centre,
    against the oracle's brute-force composite."""
    cam = object_camera(13, 7)
    rng = np.random.default_rng(1)
    M = 40
    means = (rng.normal(0, 0.05, (M, 3)) + [0, 0, -1.0]).astype(np.float32)
    gs = GaussianSet(means, rng.normal(np.log(0.01), 0.2, (M, 3)).astype(np.float32),
                     rng.normal(size=(M, 4)).astype(np.float32), rng.normal(size=M).astype(np.float32),
                     rng.uniform(size=(M, 3)).astype(np.float32))
    Ct = rng.uniform(size=(3, 7, 13)).astype(np.float32)
    Dt = np.full((7, 13), 1.7, np.float32)
    tgt = rng.uniform(size=(3, 7, 13)).astype(np.float32)
    c, d, wg, L, _ = _render(gs, cam, Ct, Dt, tgt, Dt, tile=tile, eps_depth=0.01)
    rec, _ = oracle.project(gs.astype(np.float64), cam)
    out = oracle.composite(rec, Ct, Dt, 0.01, oracle.OIT, brute=True)
    assert out["W"].max() > 0.1
    # per pixel: 1e-4 plus the oracle's envelope of decisions within the FP32 bands
    env = oracle.envelope(rec, Ct, Dt, 0.01, oracle.OIT, tgt, Dt, 0.0, 1)
    ok = env["unbounded"] == 0
    assert ok.all()
    assert np.all(np.abs(c - out["C"]).max(0) <= 1e-4 + env["allow_C"])
    assert np.all(np.abs(wg - out["W"]) <= 1e-4 + env["allow_W"])


def test_one_gaussian_covering_the_whole_image():
    """One large Gaussian: every tile lists it.  The default pair capacity (16
    entries per Gaussian) is too small and the overflow is reported; with
    room for its entries it renders like the oracle."""
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    gs = GaussianSet(np.array([[0.0, 0.0, -0.8]], np.float32), np.full((1, 3), np.log(0.4), np.float32),
                     np.array([[1.0, 0, 0, 0]], np.float32), np.array([2.0], np.float32),
                     np.array([[0.9, 0.1, 0.2]], np.float32))
    r = gps.Renderer(1, [f.cam], gps.settings(tile=(16, 8), eps_depth=1.0))
    r.forward(gps.Gaussians.from_numpy(gs), [gps.View(f.cam, cuda(Ct), cuda(Dt))])
    assert r.status() == gps.GPS_ERR_CAPACITY
    c, d, wg, L, grads = _render(gs, f.cam, Ct, Dt, f.rgb, f.depth, tile=(16, 8), eps_depth=1.0,
                                 pair_capacity=4096)
    rec, _ = oracle.project(gs.astype(np.float64), f.cam)
    out = oracle.composite(rec, Ct, Dt, 1.0, oracle.OIT)
    assert (out["W"] > 0).mean() > 0.9
    np.testing.assert_allclose(c, out["C"], atol=1e-4)
    g = {k: t.cpu().numpy() for k, t in zip(("means", "log_scales", "quats", "opacity_logits",
                                             "rgb"), grads.tensors())}
    ref = oracle.render_loss_grads(gs.astype(np.float64), f.cam, Ct, Dt, f.rgb, f.depth,
                                   eps=1.0)["grads"]
    for k in g:
        np.testing.assert_allclose(g[k], ref[k], rtol=2e-3, atol=1e-4 * np.abs(ref[k]).max())


@pytest.mark.parametrize("tile,size", [((16, 16), None), ((16, 8), None), ((8, 8), None),
                                       ((32, 8), None), ((8, 8), (1280, 720))])
def test_sort_free_default_equals_deterministic_order(tile, size):
    """The OIT blend is order-independent: the sort-free default and
    deterministic mode's lists (ascending index, fixed-order emission; at
    1280x720 with 8x8 tiles, 14,400 tiles, depth-sorted super-tile lists
    with the forward's depth cut) give the same images up to FP32 summation
    order, the same loss, and gradients that agree under the same upstream
    gradients."""
    w = workload("grad") if size is None else workload("grad", width=size[0], height=size[1])
    f = w.frames[0]
    H, W = f.cam.height, f.cam.width
    Ct, Dt, _, _ = oracle_sdf_images(w)
    up = np.sign(np.random.default_rng(2).normal(size=(3, H, W))).astype(np.float32) * 1e-3
    outs = []
    for det in (False, True):
        # the 1280x720 view's Gaussians cover many tiles each: room for all entries
        s = gps.settings(eps_depth=w.eps_depth, tile=tile, deterministic=det,
                         pair_capacity=0 if size is None else 64 * w.gaussians.M)
        r = gps.Renderer(w.gaussians.M, [f.cam], s)
        g = gps.Gaussians.from_numpy(w.gaussians)
        v = gps.View(f.cam, cuda(Ct), cuda(Dt), grad_rgb=cuda(up),
                     grad_depth=torch.zeros(H, W, device="cuda"),
                     out_rgb=torch.empty(3, H, W, device="cuda"),
                     out_weight=torch.empty(H, W, device="cuda"))
        r.forward(g, [v])
        grads = g.zeros_like()
        r.backward(g, [v], grads)
        torch.cuda.synchronize()
        assert r.status() == gps.GPS_OK
        outs.append((v.out_rgb.cpu().numpy(), v.out_weight.cpu().numpy(), grads.flat().cpu().numpy()))
    (c0, w0, g0), (c1, w1, g1) = outs
    np.testing.assert_allclose(c0, c1, atol=2e-6)
    np.testing.assert_allclose(w0, w1, rtol=2e-6, atol=2e-6)
    scale = np.abs(g1).max()
    assert np.all(np.abs(g0 - g1) <= 1e-4 * scale + 1e-4 * np.abs(g1))


@pytest.mark.parametrize("mode,tile,size", [(gps.BLEND_OIT, (16, 8), (320, 240)),
                                            (gps.BLEND_ALPHA, (16, 8), (320, 240)),
                                            (gps.BLEND_ALPHA, (8, 8), (150, 100)),
                                            (gps.BLEND_OIT, (32, 8), (150, 100))])
def test_tile_order_is_a_permutation(mode, tile, size):
    """The composites take their tiles in the order the scan writes
    (decreasing list length, in half-octave buckets): every tile exactly once,
    with bins that are the tiles themselves or super-tiles of several tiles
    (partial ones at the image edge), and bucket by bucket non-increasing in
    list length."""
    w = workload("small", M=4000, width=size[0], height=size[1])
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    s = gps.settings(eps_depth=w.eps_depth, blend_mode=mode, tile=tile)
    r = gps.Renderer(w.gaussians.M, [f.cam], s)
    g = gps.Gaussians.from_numpy(w.gaussians)
    r.forward(g, [gps.View(f.cam, cuda(Ct), cuda(Dt), cuda(f.rgb), cuda(f.depth))])
    torch.cuda.synchronize()
    assert r.status() == gps.GPS_OK
    L = r.layout(0)
    n = L.tiles_x * L.tiles_y
    order = r.region(0, "tile_order", torch.int32, n).cpu().numpy()
    np.testing.assert_array_equal(np.sort(order), np.arange(n))
    ranges = r.region(0, "tile_ranges", torch.int32, 2 * n).view(n, 2).cpu().numpy()
    if L.tile_bins:
        length = (ranges[:, 1] - ranges[:, 0]).astype(np.int64)
        # the buckets are half octaves: a later tile is at most ~1.5x longer
        lo = length[order]
        for a in range(n - 1):
            assert lo[a + 1] <= max(1, 2 * lo[a]), (a, lo[a], lo[a + 1])
