"""render_forward_noalloc: the forward pass for callers that may not allocate
device memory (for example code living inside a host application that owns
every device allocation, or a real-time loop whose memory is fixed at start-up)
runs on the library's static device scratch instead of a caller workspace.

It must give the same images and loss as render_forward with a caller-allocated
workspace, call after call (the static array keeps the previous call's
contents), and reject problems too large for the array before launching
anything.  Collected last so that a run stopping at the first failure has run
every other test already; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from datagen import workloads

pytestmark = pytest.mark.gpu


def _inputs(w):
    f = w.frames[0]
    vol = oracle.Volume(w.tsdf)
    oracle.fuse(vol, f.depth, f.rgb, f.cam)
    Ct, Dt, _, _ = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    return f, cu(Ct), cu(Dt), cu(f.rgb), cu(f.depth)


def _view(f, Ct, Dt, C, D):
    H, W = f.cam.height, f.cam.width
    return gps.View(f.cam, Ct, Dt, C, D, out_rgb=torch.empty(3, H, W, device="cuda"),
                    out_depth=torch.empty(H, W, device="cuda"),
                    out_weight=torch.empty(H, W, device="cuda"))


@pytest.mark.parametrize("mode", [gps.BLEND_OIT, gps.BLEND_ALPHA])
def test_noalloc_matches_workspace_forward_twice(mode):
    from paper_2509_11574_b300 import build
    build.build()
    L = gps.lib()
    w = workloads.small(M=2000)
    f, Ct, Dt, C, D = _inputs(w)
    s = gps.settings(eps_depth=w.eps_depth, blend_mode=mode)
    g = gps.Gaussians.from_numpy(w.gaussians)
    # reference: caller-allocated workspace
    r = gps.Renderer(g.M, [f.cam], s)
    vr = _view(f, Ct, Dt, C, D)
    loss_r = torch.zeros(1, device="cuda")
    r.forward(g, [vr], loss_r)
    torch.cuda.synchronize()
    assert gps.gps_workspace_size(g.M, [f.cam], s) <= gps.NOALLOC_SCRATCH_BYTES
    for call in range(2):
        vn = _view(f, Ct, Dt, C, D)
        loss_n = torch.zeros(1, device="cuda")
        gc = g.c()
        views = (gps.GpsView * 1)(vn.c())
        rc = L.render_forward_noalloc(ctypes.byref(gc), views, 1, ctypes.byref(s),
                                      ctypes.c_void_p(loss_n.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == gps.GPS_OK, L.gps_last_error()
        torch.cuda.synchronize()
        # same kernels, same inputs: the tolerance of the staged parity tests
        np.testing.assert_allclose(vn.out_rgb.cpu().numpy(), vr.out_rgb.cpu().numpy(), atol=1e-5)
        np.testing.assert_allclose(vn.out_depth.cpu().numpy(), vr.out_depth.cpu().numpy(),
                                   rtol=1e-5)
        np.testing.assert_allclose(vn.out_weight.cpu().numpy(), vr.out_weight.cpu().numpy(),
                                   rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(loss_n.item(), loss_r.item(), rtol=1e-6)
        st = ctypes.c_int32(-99)
        assert L.gps_noalloc_query_status(ctypes.byref(st), None) == gps.GPS_OK
        assert st.value == gps.GPS_OK


def test_noalloc_reports_pair_capacity_overflow():
    """A pair capacity too small for the frame: the overflow lands in the
    static array's status word, read back through gps_noalloc_query_status;
    the next call that fits clears it."""
    L = gps.lib()
    w = workloads.small(M=2000)
    f, Ct, Dt, C, D = _inputs(w)
    g = gps.Gaussians.from_numpy(w.gaussians)
    for cap, expect in ((64, gps.GPS_ERR_CAPACITY), (0, gps.GPS_OK)):
        s = gps.settings(eps_depth=w.eps_depth, pair_capacity=cap)
        vn = _view(f, Ct, Dt, C, D)
        gc = g.c()
        views = (gps.GpsView * 1)(vn.c())
        rc = L.render_forward_noalloc(ctypes.byref(gc), views, 1, ctypes.byref(s), None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == gps.GPS_OK, L.gps_last_error()
        st = ctypes.c_int32(-99)
        rc = L.gps_noalloc_query_status(ctypes.byref(st),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == gps.GPS_OK, L.gps_last_error()
        assert st.value == expect, (cap, st.value)


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    L = gps.lib()
    w = workloads.small(M=64)
    f = w.frames[0]
    s = gps.settings(eps_depth=w.eps_depth)
    M = 5_000_000  # records alone need 320 MB
    assert gps.gps_workspace_size(M, [f.cam], s) > gps.NOALLOC_SCRATCH_BYTES
    fake = ctypes.c_void_p(256)
    big = gps.GpsGaussians(fake, fake, fake, fake, fake, M)
    view = (gps.GpsView * 1)(gps.GpsView(gps.intrinsics(f.cam), gps.pose(f.cam), fake, fake))
    rc = L.render_forward_noalloc(ctypes.byref(big), view, 1, ctypes.byref(s), None, None)
    assert rc == gps.GPS_ERR_WORKSPACE_TOO_SMALL
    assert b"static scratch" in L.gps_last_error()
