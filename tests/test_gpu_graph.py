"""The form the bench times: one CUDA graph per frame holding fuse_frame,
raycast_sdf and 10 x (render_forward + render_backward_adam with the device
step counter), on the room workload (640x480, 100k Gaussians, 256^3 TSDF,
16x8 tiles), through bench.GpuPipeline.

  * Replayed graphs against the same C-ABI calls made eagerly, two frames in
    a row: in deterministic mode every byte of the state (volume, C_t, D_t,
    parameters, Adam moments, losses, step counter) is equal; with the
    sort-free default the volume and the ray-cast images are equal (no
    atomics there), the step counter advances by 10 per frame, and the
    losses agree to the sort-free lists' summation order.
  * The graph's first iteration against the FP64 oracle (fed the oracle's
    own fusion + ray-cast of the frame): loss, the gradient read back from
    Adam's first moment (m = (1 - beta1) g at step 1) under the oracle's
    decision envelope, and the parameter step (Adam's first step moves each
    parameter by lr sign(g); where the envelope leaves the sign open, by at
    most lr).
Later iterations are the same kernels replayed (bitwise equal to the eager
calls in deterministic mode, each eager call checked against the oracle by
the parity tests): an FP64 loop of 10 Adam steps is not compared element by
element, since Adam's first steps move every parameter by about lr whatever
the size of its gradient, so a gradient element inside its envelope of zero
may legitimately step either way and the trajectories part by ~2 lr there."""
import functools
import os
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from datagen import workloads
from helpers import (assert_grads_in_envelope, assert_record_bounds, envelope_slack,
                     gaussians_over, oracle_sdf_images, projection_skip)

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_11574_b300 import build
    build.build()
    gps.lib()


@functools.lru_cache(maxsize=1)
def _room():
    return workloads.room(n_frames=2, M=100_000)


def _pipe(det):
    return bench.GpuPipeline(_room(), (16, 8), "oit", torch.device("cuda", 0), deterministic=det)


def _state(pipe):
    torch.cuda.synchronize()
    out = {"params": pipe.g.flat().cpu().numpy(), "m": pipe.opt.m.flat().cpu().numpy(),
           "v": pipe.opt.v.flat().cpu().numpy(), "loss": pipe.loss.cpu().numpy(),
           "step": int(pipe.opt.device_step.item()), "Ct": pipe.Ct.cpu().numpy(),
           "Dt": pipe.Dt.cpu().numpy()}
    for k, t in zip(("sdf", "weight", "rgbw"), pipe.vol.linear()):
        out[k] = t.cpu().numpy()
    assert pipe.r.status() == gps.GPS_OK
    return out


@pytest.mark.parametrize("det", [True, False])
def test_graph_replay_equals_eager_calls(det):
    pipe = _pipe(det)
    for k in range(2):
        pipe.capture(k)
    pipe.reset()
    replayed = []
    for k in range(2):
        pipe.graphs[k].replay()
        replayed.append(_state(pipe))
    pipe.reset()
    eager = []
    for k in range(2):
        pipe.step(k)
        eager.append(_state(pipe))
    for k, (A, B) in enumerate(zip(replayed, eager)):
        assert A["step"] == B["step"] == 10 * (k + 1)
        for name in ("sdf", "weight", "rgbw", "Ct", "Dt"):
            np.testing.assert_array_equal(A[name], B[name], err_msg=name)
        if det:
            for name in ("params", "m", "v", "loss"):
                np.testing.assert_array_equal(A[name], B[name], err_msg=name)
        else:
            # the same kernels; the sort-free lists sum in the binning's
            # emission order, which varies from run to run
            np.testing.assert_allclose(A["loss"], B["loss"], rtol=1e-5)
        assert np.all(np.isfinite(A["params"]))
    # the optimisation ran: parameters moved and the loss fell over a frame
    assert np.abs(replayed[0]["params"] - pipe.g0.flat().cpu().numpy()).max() > 0
    assert replayed[0]["loss"][-1] < replayed[0]["loss"][0]


@pytest.mark.parametrize("det", [True, False])
def test_graph_first_iteration_matches_oracle(det):
    w = _room()
    f = w.frames[0]
    H, W = f.cam.height, f.cam.width
    g64 = w.gaussians.astype(np.float64)
    Ct, Dt, _, _ = oracle_sdf_images(w)
    ref = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                   lambda_depth=w.lambda_depth)
    pipe = _pipe(det)
    # the oracle's C_t, D_t in place of the graph's own fusion + ray-cast
    pipe.capture(0, iters=1, sdf=False)
    pipe.reset()
    pipe.Ct.copy_(torch.from_numpy(Ct))
    pipe.Dt.copy_(torch.from_numpy(Dt))
    p0 = pipe.g.flat().cpu().numpy().astype(np.float64)
    pipe.graphs[0].replay()
    st = _state(pipe)
    assert st["step"] == 1
    rec, pamb = ref["rec"], ref["proj_amb"]
    vis = (rec[:, oracle.R_VIS] > 0) & (pamb == 0)
    rec_g = pipe.r.region(0, "records", torch.float32, pipe.r.M * 16).view(pipe.r.M, 16).cpu().numpy()
    assert_record_bounds(rec_g, rec, vis, W, H, label="graph records")
    skip, excl = projection_skip(rec, pamb, H, W)
    JT = oracle.projection_adjoint_matrix(g64, f.cam)
    env = oracle.envelope(rec, Ct, Dt, w.eps_depth, oracle.OIT, f.rgb, f.depth, w.lambda_depth,
                          ref["n_valid"], JT)
    excl |= gaussians_over(env["unbounded"] != 0, rec)
    assert abs(st["loss"][0] - ref["L"]) <= 1e-4 * ref["L"] + env["allow_L"]
    # Adam's first moment after one step: m = fl((1 - beta1) g), 1 - beta1
    # taken in float as the kernel does
    M = w.gaussians.M
    sizes = [3, 3, 4, 1, 3]
    keys = ["means", "log_scales", "quats", "opacity_logits", "rgb"]
    offs = np.cumsum([0] + [M * s for s in sizes])
    g_gpu = st["m"].astype(np.float64) / np.float64(np.float32(1) - np.float32(0.9))
    got = {k: g_gpu[offs[i]:offs[i + 1]].reshape(ref["grads"][k].shape) for i, k in enumerate(keys)}
    stats = assert_grads_in_envelope(got, ref["grads"], env, JT, rec, excl, g64, f.cam,
                                     label=f"graph first iteration det={det}")
    print("graph first iteration", stats)
    # the parameter step, lr sign(g), where the gradient's tolerance interval
    # excludes zero and |g| >> eps = 1e-15 (parameters group by group, as
    # Gaussians.flat())
    slack = envelope_slack(env, JT, rec, g64, f.cam)
    cols = np.cumsum([0] + sizes)
    flat = lambda a: np.concatenate([a[:, cols[i]:cols[i + 1]].reshape(-1) for i in range(5)])
    o = np.concatenate([ref["grads"][k].reshape(-1) for k in keys])
    lr = np.concatenate([np.full(M * s, gps.LR_APP_C[i]) for i, s in enumerate(sizes)])
    ex = flat(np.repeat(excl[:, None], cols[-1], axis=1))
    sure = (np.abs(o) > 1e-4 * np.abs(o) + flat(slack)) & (np.abs(o) > 1e-10) & ~ex
    step = st["params"].astype(np.float64) - p0
    ulp = np.spacing(np.abs(p0).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(step + lr * np.sign(o))[sure] <= 2 * ulp[sure] + 2e-5 * lr[sure])
    assert np.all(np.abs(step) <= lr * (1 + 2e-5) + 2 * ulp)
    print("graph first step: sign fixed by the envelope for", float(sure.mean()), "of the parameters")
