"""View-dependent colour (SH of degree 1-3) on the GPU against the FP64
oracle: projected colours, the projection adjoint given identical 2D
gradients, the whole forward + backward, Adam's SH group, insertion and
removal of SH rows, and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from oracle import edit
import paper_2509_11574_b300 as gps
from datagen import GaussianSet
from datagen.scenes import with_sh
from helpers import assert_projection_adjoint, cuda, oracle_sdf_images, workload

pytestmark = pytest.mark.gpu


def _sh_set(name, degree, seed=5, scale=0.2):
    return with_sh(workload(name).gaussians, degree, seed=seed, scale=scale)


def _renderer(w, gs, cams, **kw):
    s = gps.settings(eps_depth=w.eps_depth, lambda_depth=w.lambda_depth, near=w.near, **kw)
    return gps.Renderer(gs.M, cams, s)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_projected_colour_matches_oracle(degree):
    w = workload("grad")
    f = w.frames[0]
    gs = _sh_set("grad", degree)
    Ct, Dt, _, _ = oracle_sdf_images(w)
    rec_o, amb = oracle.project(gs.astype(np.float64), f.cam)
    r = _renderer(w, gs, [f.cam], stages=gps.STAGE_PROJECT)
    g = gps.Gaussians.from_numpy(gs)
    assert g.sh_degree == degree
    r.forward(g, [gps.View(f.cam, cuda(Ct), cuda(Dt))])
    rec_g = r.region(0, "records", torch.float32, r.M * 16).view(r.M, 16).cpu().numpy()
    both = (rec_o[:, oracle.R_VIS] > 0) & (rec_g[:, 11] >= 0) & (amb == 0)
    assert both.sum() > 1000
    col_o = rec_o[both][:, [oracle.R_R, oracle.R_G, oracle.R_B]]
    col_g = rec_g[both][:, 8:11].astype(np.float64)
    # FP32: a few ulps of the terms (|Y f| <= ~1)
    np.testing.assert_allclose(col_g, col_o, atol=2e-6)
    # the SH terms really move the colour away from rgb
    assert np.abs(col_o - gs.rgb[both]).max() > 0.05


@pytest.mark.parametrize("degree", [1, 3])
def test_projection_backward_with_sh_staged(degree):
    """Identical 2D gradients in: means (now also through the view direction),
    rgb and SH coefficient gradients out."""
    w = workload("grad")
    f = w.frames[0]
    gs = _sh_set("grad", degree)
    Ct, Dt, _, _ = oracle_sdf_images(w)
    g64 = gs.astype(np.float64)
    rng = np.random.default_rng(3)
    g2 = rng.normal(size=(gs.M, 10)).astype(np.float32)
    rec_o, amb = oracle.project(g64, f.cam)
    g2 = np.where((rec_o[:, oracle.R_VIS] > 0)[:, None], g2, 0).astype(np.float32)
    ref = oracle.project_backward(g64, f.cam, g2.astype(np.float64))
    r = _renderer(w, gs, [f.cam], stages=gps.STAGE_PROJECT_BWD)
    g2pad = np.zeros((gs.M, 12), np.float32)
    g2pad[:, :10] = g2
    r.region(0, "grad2d", torch.float32, r.M * 12).copy_(torch.from_numpy(g2pad.reshape(-1)).cuda())
    g = gps.Gaussians.from_numpy(gs)
    v = gps.View(f.cam, cuda(Ct), cuda(Dt), grad_rgb=cuda(np.zeros_like(Ct)))
    grads = g.zeros_like()
    r.backward(g, [v], grads)
    got = {k: t.cpu().numpy() for k, t in zip(ref.keys(), grads.tensors())}
    assert set(ref) == {"means", "log_scales", "quats", "opacity_logits", "rgb", "sh_rest"}
    vis = (rec_o[:, oracle.R_VIS] > 0) & (amb == 0)
    worst = assert_projection_adjoint(got, ref, g64, f.cam, g2, rec_o, vis,
                                      label="project_backward_sh")
    print("project_backward_sh: worst error / bound", worst)


@pytest.mark.parametrize("name,degree", [("small", 3), ("grad", 2)])
def test_end_to_end_with_sh(name, degree):
    """Projection, binning, composite, fused loss and backward with SH colour
    vs the oracle, under the same tolerances and allowances as without SH."""
    from test_gpu_parity import _end_to_end
    w = workload(name)
    _end_to_end(w, gps.BLEND_OIT, lam=w.lambda_depth, gs=_sh_set(name, degree))


def test_adam_sh_group_matches_oracle():
    rng = np.random.default_rng(0)
    M = 1001
    gs = GaussianSet(rng.normal(size=(M, 3)), rng.normal(size=(M, 3)), rng.normal(size=(M, 4)),
                     rng.normal(size=M), rng.uniform(size=(M, 3)),
                     sh_rest=rng.normal(size=(M, 8, 3))).astype(np.float32)
    p = gps.Gaussians.from_numpy(gs)
    opt = gps.Adam(p)
    ref = [a.astype(np.float64).copy() for a in gs.arrays()] + [gs.sh_rest.astype(np.float64)]
    lrs = list(gps.LR_APP_C) + [gps.LR_SH_REST]
    m = [np.zeros_like(a) for a in ref]
    vv = [np.zeros_like(a) for a in ref]
    for step in range(1, 4):
        gr = [rng.normal(size=a.shape).astype(np.float32) for a in ref]
        grads = gps.Gaussians(*[torch.from_numpy(x).cuda() for x in gr])
        opt.step(grads)
        for k in range(6):
            oracle.adam(ref[k].reshape(-1), gr[k].astype(np.float64).reshape(-1), m[k].reshape(-1),
                        vv[k].reshape(-1), lrs[k], 0.9, 0.999, 1e-15, step)
        assert float(grads.flat().abs().max()) == 0.0
    for k, t in enumerate(p.tensors()):
        np.testing.assert_allclose(t.cpu().numpy(), ref[k], rtol=1e-6, atol=1e-6 * lrs[k])


def _device_set(cap, K):
    z = lambda *s: torch.zeros(*s, device="cuda")
    return gps.Gaussians(z(cap, 3), z(cap, 3), z(cap, 4), z(cap), z(cap, 3), z(cap, K, 3))


def test_removal_and_insertion_carry_sh_rows():
    rng = np.random.default_rng(2)
    M, K = 3000, 15
    g = _device_set(M, K)
    m, v, gr = _device_set(M, K), _device_set(M, K), _device_set(M, K)
    ls = np.log(rng.uniform(0.001, 0.2, size=(M, 3))).astype(np.float32)
    lg = rng.normal(0, 3, size=M).astype(np.float32)
    sh = rng.normal(size=(M, K, 3)).astype(np.float32)
    g.log_scales.copy_(torch.from_numpy(ls))
    g.opacity_logits.copy_(torch.from_numpy(lg))
    g.sh_rest.copy_(torch.from_numpy(sh))
    for z in (m, v, gr):
        z.sh_rest.copy_(torch.from_numpy(sh) * 2)
    keep = edit.removal_keep(ls, lg)
    assert 0 < keep.sum() < M
    s = gps.edit_settings()
    scratch = torch.zeros(gps.gps_edit_scratch_size(M, 1, 1), dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    gps.remove_gaussians(g, M, m, v, gr, s, scratch, count)
    n = int(count.item())
    assert n == keep.sum()
    np.testing.assert_array_equal(g.sh_rest[:n].cpu().numpy(), sh[keep])
    np.testing.assert_array_equal(m.sh_rest[:n].cpu().numpy(), 2 * sh[keep])
    assert float(gr.sh_rest[n:].abs().max()) == 0.0     # moment / gradient tails cleared
    np.testing.assert_array_equal(g.log_scales[:n].cpu().numpy(), ls[keep])
    # insertion appends Gaussians whose SH coefficients and moments start at zero
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    vol = oracle.Volume(w.tsdf)
    oracle.fuse(vol, f.depth, f.rgb, f.cam)
    _, _, V, _ = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
    H, W = f.cam.height, f.cam.width
    for z in (g, m, v, gr):
        z.sh_rest[n:].fill_(7.0)
    scratch = torch.zeros(gps.gps_edit_scratch_size(M, W, H), dtype=torch.uint8, device="cuda")
    gps.insert_gaussians(g, n, m, v, gr, f.cam, cuda(V), cuda(Dt), cuda(Ct),
                         torch.zeros(H, W, device="cuda"), cuda(f.rgb), s, scratch, count)
    n2 = int(count.item())
    assert n2 > n
    for z in (g, m, v, gr):
        assert float(z.sh_rest[n:n2].abs().max()) == 0.0
        assert float(z.sh_rest[n2:].min()) == 7.0           # rows past the count untouched
    np.testing.assert_array_equal(g.sh_rest[:n].cpu().numpy(), sh[keep])


def test_autograd_with_sh_matches_render_backward():
    w = workload("small")
    f = w.frames[0]
    gs = _sh_set("small", 2)
    Ct, Dt, _, _ = oracle_sdf_images(w)
    s = gps.settings(eps_depth=w.eps_depth, deterministic=True)
    r = gps.Renderer(gs.M, [f.cam], s)
    g = gps.Gaussians.from_numpy(gs)
    params = [t.clone().requires_grad_(True) for t in g.tensors()]
    v = gps.View(f.cam, cuda(Ct), cuda(Dt), cuda(f.rgb), cuda(f.depth))
    loss = gps.RenderLoss.apply(r, [v], *params)
    loss.backward()
    grads = g.zeros_like()
    l2 = torch.zeros(1, device="cuda")
    r.forward(g, [v], l2)
    r.backward(g, [v], grads)
    assert abs(loss.item() - l2.item()) <= 1e-6 * abs(l2.item())
    for p, t in zip(params, grads.tensors()):
        assert torch.equal(p.grad, t)
    assert float(params[5].grad.abs().max()) > 0
