"""Gaussian insertion and removal (Sec. 3.2, App. A) on the GPU against the
numpy oracle (oracle/edit.py) on the same inputs: which pixels receive a
Gaussian and which Gaussians are removed must agree exactly (integer
decisions taken in float32 on both sides); the new parameters to float32
rounding of the window search and the normal."""
import numpy as np
import pytest
import torch

import oracle
from oracle import edit
import paper_2509_11574_b300 as gps
from helpers import cuda, oracle_sdf_images, workload

pytestmark = pytest.mark.gpu


def _frame_inputs(w):
    """C_t, D_t, V from the oracle ray-cast; C*, W_G from the oracle composite
    of the workload's Gaussians (rounded to float32)."""
    f = w.frames[0]
    vol = oracle.Volume(w.tsdf)
    oracle.fuse(vol, f.depth, f.rgb, f.cam)
    Ct, Dt, V, _ = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
    rec, _ = oracle.project(w.gaussians.astype(np.float64), f.cam)
    out = oracle.composite(rec, Ct, Dt, w.eps_depth, oracle.OIT)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    return f, f32(Dt), f32(V), f32(out["C"]), f32(out["W"]), f32(f.rgb)


def _device_set(M_cap, src=None, M=0):
    g = gps.Gaussians(torch.zeros(M_cap, 3, device="cuda"), torch.zeros(M_cap, 3, device="cuda"),
                      torch.zeros(M_cap, 4, device="cuda"), torch.zeros(M_cap, device="cuda"),
                      torch.zeros(M_cap, 3, device="cuda"))
    if src is not None:
        for t, a in zip(g.tensors(), src.arrays()):
            t[:M] = torch.as_tensor(np.asarray(a, np.float32)).cuda()
    return g


@pytest.mark.parametrize("extra", [100000, 7])
def test_insertion_matches_oracle(extra):
    w = workload("small")
    f, Dt, V, Cs, WG, Ck = _frame_inputs(w)
    M = w.gaussians.M
    cap = M + extra
    seed = 12345
    ref, pix, mask = edit.insert(V.astype(np.float64), Dt, Cs, WG, Ck, f.cam.fx,
                                 np.asarray(f.cam.t, np.float64), seed, M, cap)
    assert mask.sum() > 200 and len(edit.sampled_pixels(mask, seed)) > 50
    g = _device_set(cap, w.gaussians, M)
    m, v = _device_set(cap), _device_set(cap)
    for t in m.tensors() + v.tensors():
        t.fill_(7.0)  # must be zeroed for the new rows
    s = gps.edit_settings(seed=seed)
    scratch = torch.zeros(gps.gps_edit_scratch_size(cap, f.cam.width, f.cam.height),
                          dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    gps.insert_gaussians(g, M, m, v, None, f.cam, cuda(V), cuda(Dt), cuda(Cs), cuda(WG),
                         cuda(Ck), s, scratch, count)
    n_new = int(count.item()) - M
    assert n_new == len(pix) == min(extra, len(edit.sampled_pixels(mask, seed)))
    sl = slice(M, M + n_new)
    got = {k: t[sl].cpu().numpy().astype(np.float64) for k, t in
           zip(("means", "log_scales", "quats", "opacity_logits", "rgb"), g.tensors())}
    # copies: exact (the oracle's values are float32 inputs)
    np.testing.assert_array_equal(got["means"], ref["means"])
    np.testing.assert_array_equal(got["rgb"], ref["rgb"])
    assert np.all(got["opacity_logits"] == 0.0)
    # float32 distances, square root and logarithm
    np.testing.assert_allclose(got["log_scales"], ref["log_scales"], atol=2e-6)
    # float32 cross product of vertex differences: the same rotation within
    # 1e-3 rad (|<q, q'>| = cos of half the angle between the two rotations)
    dots = np.abs(np.sum(got["quats"] * ref["quats"], 1))
    assert np.all(dots > np.cos(0.5e-3)), dots.min()
    # the old rows are untouched, the new rows of the moments zeroed
    np.testing.assert_array_equal(g.means[:M].cpu().numpy(), w.gaussians.means.astype(np.float32))
    for t in m.tensors() + v.tensors():
        assert torch.all(t[sl] == 0) and torch.all(t[:M] == 7.0)


def test_removal_matches_oracle():
    rng = np.random.default_rng(4)
    M, cap = 5000, 6000
    gs = workload("small", M=M).gaussians.astype(np.float32)
    ls = gs.log_scales.copy()
    ls[rng.random(M) < 0.1] += 3.0           # some too large
    ls[rng.random(M) < 0.1] -= 2.5           # some too small
    lg = gs.opacity_logits.copy()
    lg[rng.random(M) < 0.1] = -6.0           # some nearly transparent
    from datagen import GaussianSet
    src = GaussianSet(gs.means, ls, gs.quats, lg, gs.rgb)
    keep = edit.removal_keep(ls, lg)
    assert 0.5 * M < keep.sum() < 0.9 * M
    g = _device_set(cap, src, M)
    mom = [rng.normal(size=a.shape).astype(np.float32) for a in src.arrays()]
    m = _device_set(cap, GaussianSet(*mom), M)
    v = _device_set(cap, GaussianSet(*[a * 2 for a in mom]), M)
    scratch = torch.zeros(gps.gps_edit_scratch_size(cap, 0, 0), dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    gps.remove_gaussians(g, M, m, v, None, gps.edit_settings(), scratch, count)
    kept = int(count.item())
    assert kept == keep.sum()
    for t, a in zip(g.tensors(), src.arrays()):
        np.testing.assert_array_equal(t[:kept].cpu().numpy(), np.asarray(a, np.float32)[keep])
    for t, a in zip(m.tensors(), mom):
        np.testing.assert_array_equal(t[:kept].cpu().numpy(), a[keep])
        assert torch.all(t[kept:M] == 0)
    for t, a in zip(v.tensors(), mom):
        np.testing.assert_array_equal(t[:kept].cpu().numpy(), 2 * a[keep])
