"""The adjoint behind torch.autograd: RenderLoss and RenderImages give the
C ABI's gradients, match the FP64 oracle's adjoint, and match central finite
differences of the GPU forward itself on parameters whose perturbation leaves
every counting decision unchanged."""
import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from datagen.scenes import GaussianSet
from helpers import (assert_grads_close, assert_grads_in_envelope, cuda, gaussians_over,
                     oracle_sdf_images, projection_skip, workload)

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "rgb")


def _params(w):
    g = gps.Gaussians.from_numpy(w.gaussians)
    return [t.clone().requires_grad_(True) for t in g.tensors()]


def test_render_loss_function_equals_the_c_abi():
    w = workload("small")
    f = w.frames[0]
    Ct, Dt, _, _ = oracle_sdf_images(w)
    s = gps.settings(eps_depth=w.eps_depth, lambda_depth=1.0, deterministic=True)
    v = gps.View(f.cam, cuda(Ct), cuda(Dt), cuda(f.rgb), cuda(f.depth))
    ps = _params(w)
    r = gps.Renderer(w.gaussians.M, [f.cam], s)
    loss = gps.RenderLoss.apply(r, [v], *ps)
    (2.0 * loss).backward()  # the upstream 2 goes in as *dloss
    g = gps.Gaussians.from_numpy(w.gaussians)
    r2 = gps.Renderer(w.gaussians.M, [f.cam], s)
    l2 = torch.zeros(1, device="cuda")
    r2.forward(g, [v], l2)
    grads = g.zeros_like()
    r2.backward(g, [v], grads, torch.full((1,), 2.0, device="cuda"))
    assert loss.item() == l2.item()
    for p, t in zip(ps, grads.tensors()):
        np.testing.assert_array_equal(p.grad.cpu().numpy(), t.cpu().numpy())


def _linear_functional(H, W, seed=0):
    rng = np.random.default_rng(seed)
    wc = rng.uniform(-1, 1, size=(3, H, W)) / (H * W)
    wd = rng.uniform(-1, 1, size=(H, W)) / (H * W)
    return wc, wd


@pytest.mark.parametrize("mode", [gps.BLEND_OIT, gps.BLEND_ALPHA])
def test_render_images_function_vs_oracle_adjoint(mode):
    """L = <w_c, C*> + <w_d, D*> through RenderImages against the oracle's
    adjoint with the same upstream gradients (decisions taken in FP32 by the
    kernel and in FP64 by the oracle: the oracle's decision envelope
    applies)."""
    w = workload("small")
    f = w.frames[0]
    H, W = f.cam.height, f.cam.width
    Ct, Dt, _, _ = oracle_sdf_images(w)
    wc, wd = _linear_functional(H, W)
    g64 = w.gaussians.astype(np.float64)
    rec, pamb = oracle.project(g64, f.cam)
    ref = oracle.project_backward(g64, f.cam, oracle.composite_backward(rec, Ct, Dt, w.eps_depth,
                                                                        wc, wd, mode))
    s = gps.settings(eps_depth=w.eps_depth, blend_mode=mode)
    r = gps.Renderer(w.gaussians.M, [f.cam], s)
    ps = _params(w)
    C, D, _ = gps.RenderImages.apply(r, gps.View(f.cam, cuda(Ct), cuda(Dt)), *ps)
    L = (C * cuda(wc)).sum() + (D * cuda(wd)).sum()
    L.backward()
    assert r.status() == gps.GPS_OK
    got = {n: p.grad.cpu().numpy() for n, p in zip(NAMES, ps)}
    # the oracle's envelope of the counting decisions within the FP32 bands,
    # with these upstream gradients (no L1 sign is involved)
    JT = oracle.projection_adjoint_matrix(g64, f.cam)
    env = oracle.envelope(rec, Ct, Dt, w.eps_depth, mode, f.rgb, f.depth, 0.0, 1, JT, dC=wc, dD=wd)
    skip, excl = projection_skip(rec, pamb, H, W)
    excl |= gaussians_over(env["unbounded"] != 0, rec)
    assert_grads_in_envelope(got, ref, env, JT, rec, excl, g64, f.cam,
                             label=f"RenderImages mode={mode}")


def test_finite_differences_of_the_gpu_forward():
    """Central differences of L = <w_c, C*> + <w_d, D*> (images read back and
    summed in FP64) against RenderImages' gradient: every rgb entry of a few
    Gaussians (L is linear in rgb) and the opacity logits of Gaussians whose
    +-h perturbation leaves the oracle's per-pixel counts unchanged.  The
    differenced forwards run with deterministic mode's fixed-order lists
    (ascending index), so that both see one summation order and the
    difference holds no rounding noise from the sort-free lists' varying
    order."""
    w = workload("small")
    f = w.frames[0]
    H, W = f.cam.height, f.cam.width
    Ct, Dt, _, _ = oracle_sdf_images(w)
    wc, wd = _linear_functional(H, W, seed=1)
    s = gps.settings(eps_depth=w.eps_depth)
    r = gps.Renderer(w.gaussians.M, [f.cam], s)
    v = gps.View(f.cam, cuda(Ct), cuda(Dt))
    ps = _params(w)
    C, D, _ = gps.RenderImages.apply(r, v, *ps)
    ((C * cuda(wc)).sum() + (D * cuda(wd)).sum()).backward()
    grad = {n: p.grad.cpu().numpy().astype(np.float64) for n, p in zip(NAMES, ps)}

    r = gps.Renderer(w.gaussians.M, [f.cam], gps.settings(eps_depth=w.eps_depth, deterministic=True))
    base = gps.Gaussians.from_numpy(w.gaussians)
    view = gps.View(f.cam, cuda(Ct), cuda(Dt), out_rgb=torch.empty(3, H, W, device="cuda"),
                    out_depth=torch.empty(H, W, device="cuda"))

    def L_gpu(name, i, c, delta):
        t = getattr(base, name)
        old = t[i, c].item() if t.dim() == 2 else t[i].item()
        if t.dim() == 2:
            t[i, c] = old + delta
        else:
            t[i] = old + delta
        r.forward(base, [view])
        Cg = view.out_rgb.cpu().numpy().astype(np.float64)
        Dg = view.out_depth.cpu().numpy().astype(np.float64)
        if t.dim() == 2:
            t[i, c] = old
        else:
            t[i] = old
        return float((Cg * wc).sum() + (Dg * wd).sum())

    g64 = w.gaussians.astype(np.float64)
    rec0, _ = oracle.project(g64, f.cam)
    vis = np.nonzero(rec0[:, oracle.R_VIS] > 0)[0]
    rng = np.random.default_rng(2)
    n0 = oracle.composite(rec0, Ct, Dt, w.eps_depth)["n"]

    def same_events(i, h):
        for sgn in (-1.0, 1.0):
            gp = GaussianSet(*(a.copy() for a in g64.arrays()))
            gp.opacity_logits[i] += sgn * h
            if not np.array_equal(oracle.composite(oracle.project(gp, f.cam)[0], Ct, Dt,
                                                   w.eps_depth)["n"], n0):
                return False
        return True

    checked = 0
    # rgb: exactly linear, h = 0.05
    for i in rng.choice(vis, 4, replace=False):
        for c in range(3):
            fd = (L_gpu("rgb", i, c, 0.05) - L_gpu("rgb", i, c, -0.05)) / 0.1
            an = grad["rgb"][i, c]
            assert abs(fd - an) <= 2e-3 * abs(an) + 1e-9, ("rgb", i, c, fd, an)
            checked += 1
    # opacity logits of Gaussians with a large gradient and no event change
    cand = vis[np.argsort(-np.abs(grad["opacity_logits"][vis]))[:40]]
    h = 1e-2
    n_logit = 0
    for i in cand:
        if n_logit == 8:
            break
        if not same_events(i, h):
            continue
        fd = (L_gpu("opacity_logits", i, 0, h) - L_gpu("opacity_logits", i, 0, -h)) / (2 * h)
        an = grad["opacity_logits"][i]
        assert abs(fd - an) <= 1e-2 * abs(an) + 1e-8, ("logit", i, fd, an)
        n_logit += 1
    assert n_logit >= 4
    checked += n_logit
    assert checked >= 16
