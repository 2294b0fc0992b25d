"""render_backward_adam (render_backward + adam_step in one call, no gradient
array) against the two calls it replaces.  Where the backward is
reproducible (deterministic mode) the results agree to a few ulps: the Adam
update's roundings are spelled out in both kernels, but the projection
adjoint is compiled into two kernels whose FMA contractions are the
compiler's choice (seen: a few in a thousand moments apart by about 1e-10).  With the
sort-free default the gradient atomics run in varying order, so the bound is
FP32 summation-order noise."""
import pytest
import torch

import paper_2509_11574_b300 as gps
from datagen.scenes import with_sh
from helpers import cuda, oracle_sdf_images, workload

pytestmark = pytest.mark.gpu


def _moments(g, seed):
    # nonzero Adam state, so that every term of the update matters
    gen = torch.Generator(device="cuda").manual_seed(seed)
    m, v = g.zeros_like(), g.zeros_like()
    for t in m.tensors():
        t.copy_(torch.randn(t.shape, generator=gen, device="cuda") * 1e-3)
    for t in v.tensors():
        t.copy_(torch.rand(t.shape, generator=gen, device="cuda") * 1e-6)
    return m, v


@pytest.mark.parametrize("device_step", [False, True])
@pytest.mark.parametrize("sh_degree,det", [(0, True), (2, True), (0, False), (3, False)])
def test_fused_backward_adam_equals_backward_then_adam(sh_degree, det, device_step):
    w = workload("small")
    f = w.frames[0]
    gs = w.gaussians if sh_degree == 0 else with_sh(w.gaussians, sh_degree, seed=3, scale=0.05)
    Ct, Dt, _, _ = oracle_sdf_images(w)
    s = gps.settings(eps_depth=w.eps_depth, lambda_depth=0.5, deterministic=det)
    r = gps.Renderer(gs.M, [f.cam], s)
    view = gps.View(f.cam, cuda(Ct), cuda(Dt), cuda(f.rgb), cuda(f.depth))
    out = []
    for fused in (False, True):
        g = gps.Gaussians.from_numpy(gs)
        m, v = _moments(g, 5)
        ds = torch.full((1,), 2, dtype=torch.int32, device="cuda") if device_step else None
        step = 0 if device_step else 3
        r.forward(g, [view], torch.zeros(1, device="cuda"))
        if fused:
            gps.render_backward_adam(g, [view], s, r.ws, m, v, step=step, device_step=ds)
        else:
            grads = g.zeros_like()
            gps.render_backward(g, [view], s, r.ws, grads)
            gps.adam_step(g, grads, m, v, step=step, device_step=ds)
            assert max(float(t.abs().max()) for t in grads.tensors()) == 0.0  # zeroed by Adam
        torch.cuda.synchronize()
        assert r.status() == gps.GPS_OK
        out.append((g.tensors() + m.tensors() + v.tensors(), ds))
    (a, d0), (b, d1) = out
    assert len(a) == len(b) == 3 * (5 + (sh_degree > 0))
    moved = 0
    for n, (x, y) in enumerate(zip(a, b)):
        if det:
            torch.testing.assert_close(x, y, rtol=1e-6, atol=1e-9, msg=f"tensor {n}")
        else:
            torch.testing.assert_close(x, y, rtol=1e-4, atol=1e-7)
    # the step did something: parameters left their initial values
    g0 = gps.Gaussians.from_numpy(gs).tensors()
    for x, y in zip(a[:len(g0)], g0):
        moved += int((x != y).sum())
    assert moved > gs.M
    if device_step:
        assert int(d0) == int(d1) == 3
