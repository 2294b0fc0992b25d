"""Reduced-precision colour storage at the 1280 x 720, 1,000,000-Gaussian size
of the large room workload (5.12 m room): errors of the stored C* against the
FP64 oracle on 2 sample frames, for float, binary16 and bfloat16 storage.

Inputs are the frames themselves: C_t = the frame's colour, D_t its depth (a
stand-in for the ray-cast images, which would need a 512^3 FP64 volume on the
oracle side), targets = the same frame.  Every side takes the colour images
rounded to the storage type; the oracle reference takes them unrounded, so
the reported error is the whole storage + FP32 arithmetic error.  Counting
decisions depend on depth only (always float), so the image bound is the
FP32 one plus the rounding of C_t (through 1 / (1 + W_G)) and of the stored
C*.  Loss and gradient errors (fused L1 loss, colour term) are reported, not
bounded: a rounded target can flip the sign of an L1 residual near zero."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2509_11574_b300 as gps
from helpers import cuda, projection_skip, workload

pytestmark = pytest.mark.gpu

_U = {gps.PREC_FP32: 2.0 ** -24, gps.PREC_FP16: 2.0 ** -11, gps.PREC_BF16: 2.0 ** -8}


def _rel(got, ref):
    scale = np.abs(ref).max()
    return {"max_rel": float(np.abs(got - ref).max() / scale),
            "mean_rel": float(np.abs(got - ref).mean() / np.abs(ref).mean())}


def test_large_config_colour_precision_errors_vs_fp64(capsys):
    w = workload("room", n_frames=2, M=1_000_000, width=1280, height=720, size=5.12, n_vox=512)
    g64 = w.gaussians.astype(np.float64)
    g = gps.Gaussians.from_numpy(w.gaussians)
    report = {}
    for k, f in enumerate(w.frames):
        H, W = f.cam.height, f.cam.width
        ref = oracle.render_loss_grads(g64, f.cam, f.rgb, f.depth, f.rgb, f.depth,
                                       eps=w.eps_depth, lambda_depth=0.0, mode=oracle.OIT)
        out, rec, pamb = ref["out"], ref["rec"], ref["proj_amb"]
        skip, _ = projection_skip(rec, pamb, H, W)
        # the oracle's envelope of decisions within the FP32 bands (images only)
        env = oracle.envelope(rec, f.rgb, f.depth, w.eps_depth, oracle.OIT, f.rgb, f.depth, 0.0,
                              ref["n_valid"])
        ok = ~skip & (env["unbounded"] == 0)
        assert ok.mean() > 0.99
        for prec in (gps.PREC_FP32, gps.PREC_FP16, gps.PREC_BF16):
            cdt = gps.PREC_DTYPE[prec]
            Cq = oracle.quantise(f.rgb, prec).astype(np.float32)
            s = gps.settings(eps_depth=w.eps_depth, precision=prec, tile=(16, 8),
                             pair_capacity=32 * g.M)
            r = gps.Renderer(g.M, [f.cam], s)
            v = gps.View(f.cam, cuda(Cq).to(cdt), cuda(f.depth), cuda(Cq).to(cdt), cuda(f.depth),
                         out_rgb=torch.empty(3, H, W, device="cuda", dtype=cdt))
            loss = torch.zeros(1, device="cuda")
            r.forward(g, [v], loss)
            grads = g.zeros_like()
            r.backward(g, [v], grads)
            assert r.status() == gps.GPS_OK
            err = np.abs(v.out_rgb.float().cpu().numpy() - out["C"])
            u = _U[prec]
            Ct_part = np.abs(f.rgb) / (1.0 + out["W"])[None]
            tol = 1e-4 + env["allow_C"][None] + u * (Ct_part + np.abs(out["C"]) + 1e-4)
            assert np.all(err[:, ok] <= tol[:, ok]), (prec, (err - tol)[:, ok].max())
            got = {n: t.cpu().numpy().astype(np.float64)
                   for n, t in zip(ref["grads"].keys(), grads.tensors())}
            assert all(np.all(np.isfinite(a)) for a in got.values())
            report.setdefault({0: "fp32", 1: "fp16", 2: "bf16"}[prec], []).append(
                {"frame": k, "image": {"max_abs": float(err[:, ok].max()),
                                       "mean_abs": float(err[:, ok].mean())},
                 "loss_rel": abs(loss.item() - ref["L"]) / ref["L"],
                 "grads": {n: _rel(got[n], ref["grads"][n]) for n in got}})
    with capsys.disabled():
        print("\ncolour storage errors vs FP64 (1280x720, 1e6 Gaussians):", json.dumps(report))
