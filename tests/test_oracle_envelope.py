"""Pins of the oracle's decision envelope (`oracle.envelope`, orc_envelope in
splat.cpp): the bound the end-to-end GPU tests use for counting decisions and
L1 signs that lie within the FP32 error band of their thresholds.

Hand cases (records written directly, JT = identity so the envelope is read
in the 2D gradient's coordinates):
  * one Gaussian whose support boundary q = qmax passes exactly through four
    pixel centres;
  * one Gaussian whose depth equals D_t + eps, so every pixel of its support
    holds an ambiguous depth test;
  * a residual that is exactly zero in one channel of one pixel (free sign).
Each allowance is the range between the two decisions, computed here from
Eq. 4 and the L1 adjoint by hand.  Then: the envelope's reference gradient
is the oracle's adjoint bit for bit, zero bands give zero allowances, and on
a random scene every combination of flipped decisions the oracle can be made
to take (all inverted, and seeded coins) stays inside the envelope."""
import math

import numpy as np
import pytest

import oracle
from datagen import workloads

W9 = H9 = 9
NPX = W9 * H9
RGB = np.array([0.9, 0.6, 0.3])
CT = 0.2


def record(mx, my, d, sig, a, b, c, qmax, rgb=RGB, ext=6.0):
    r = np.zeros(oracle.R_N)
    r[[oracle.R_MX, oracle.R_MY, oracle.R_D, oracle.R_SIG]] = mx, my, d, sig
    r[[oracle.R_CA, oracle.R_CB, oracle.R_CC, oracle.R_QMAX]] = a, b, c, qmax
    r[oracle.R_R:oracle.R_B + 1] = rgb
    r[[oracle.R_EX, oracle.R_EY, oracle.R_VIS]] = ext, ext, 1.0
    return r[None]


def images(Dt=1.0, Ctgt=0.0):
    Ct = np.full((3, H9, W9), CT)
    D = np.full((H9, W9), Dt)
    Ctg = np.full((3, H9, W9), Ctgt) if np.isscalar(Ctgt) else Ctgt
    Dtg = np.ones((H9, W9))
    return Ct, D, Ctg, Dtg


def eye_jt(M=1):
    return np.tile(np.eye(oracle.G_N)[None], (M, 1, 1))


BANDS = oracle.bands_for(W9, H9)
SC = 1.0 / (3 * NPX)  # dL/dC* of one channel of one valid pixel (Eq. 6)


def terms_oit(alpha, G, rgb=RGB, ct=CT, sign=(1.0, 1.0, 1.0)):
    """By hand: one Gaussian counted alone at a pixel (Eq. 4, L1 adjoint)."""
    N = 1.0 + alpha
    Cs = (ct + alpha * rgb) / N
    g = np.asarray(sign) * SC
    dLdc = g * alpha / N
    dLda = np.sum(g * (rgb - Cs)) / N
    return Cs, dLdc, dLda * G


def test_support_boundary_through_four_pixel_centres():
    v = 2.0  # isotropic Sigma_2D = v I: q = r^2 / v, qmax = 4.5 at r = 3
    sig = math.exp(2.25) / 255.0  # alpha = 1/255 exactly on the boundary
    rec = record(4.0, 4.0, 0.5, sig, 1 / v, 0.0, 1 / v, 4.5)
    Ct, Dt, Ctg, Dtg = images()
    env = oracle.envelope(rec, Ct, Dt, 0.01, oracle.OIT, Ctg, Dtg, 0.0, NPX, eye_jt(), BANDS)
    on = np.zeros((H9, W9), bool)
    on[4, [1, 7]] = on[[1, 7], 4] = True
    np.testing.assert_array_equal(env["n_amb"] > 0, on)
    assert env["unbounded"].sum() == 0
    ab = sig * math.exp(-2.25)  # 1/255 up to rounding
    Cs, dLdc, dsig = terms_oit(ab, ab / sig)
    np.testing.assert_allclose(env["allow_C"][on], np.max(np.abs(Cs - CT)), rtol=1e-12)
    assert np.all(env["allow_C"][~on] == 0)
    np.testing.assert_allclose(env["allow_W"][on], ab, rtol=1e-12)  # W_G moves by alpha
    # per pixel the Gaussian's term lies between 0 (not counted) and its value
    a3 = env["allow3"][0]
    np.testing.assert_allclose(a3[oracle.G_R:oracle.G_B + 1], 4 * dLdc, rtol=1e-12)
    np.testing.assert_allclose(a3[oracle.G_SIG], 4 * abs(dsig), rtol=1e-12)
    np.testing.assert_allclose(env["allow_L"], 4 * np.sum(np.abs(Cs - CT)) * SC, rtol=1e-12)


def test_depth_threshold_at_every_support_pixel():
    v, sig, d, eps = 1.5, 0.6, 0.8, 0.01
    qmax = 2 * math.log(255 * sig)
    rec = record(4.2, 3.9, d, sig, 1 / v, 0.0, 1 / v, qmax)
    Ct, Dt, Ctg, Dtg = images(Dt=d - eps)  # D_t + eps = d up to one rounding
    env = oracle.envelope(rec, Ct, Dt, eps, oracle.OIT, Ctg, Dtg, 0.0, NPX, eye_jt(), BANDS)
    ys, xs = np.mgrid[0:H9, 0:W9]
    q = ((xs - 4.2) ** 2 + (ys - 3.9) ** 2) / v
    inside = q <= qmax
    assert np.all(np.abs(q - qmax) > 1e-3)  # no support decision near its threshold
    np.testing.assert_array_equal(env["n_amb"] > 0, inside)
    al = sig * np.exp(-0.5 * q[inside])
    rgb_t, sig_t = 0.0, 0.0
    for a in al:
        Cs, dLdc, dsig = terms_oit(a, a / sig)
        rgb_t = rgb_t + dLdc
        sig_t += abs(dsig)
    a3 = env["allow3"][0]
    np.testing.assert_allclose(a3[oracle.G_R:oracle.G_B + 1], rgb_t, rtol=1e-12)
    np.testing.assert_allclose(a3[oracle.G_SIG], sig_t, rtol=1e-12)
    # the depth term: dL/dd = g_D alpha / N with lambda = 0 is zero
    assert a3[oracle.G_D] == 0.0


def test_free_residual_sign_at_one_pixel():
    v, sig = 1.5, 0.6
    qmax = 2 * math.log(255 * sig)
    rec = record(4.0, 4.0, 0.5, sig, 1 / v, 0.0, 1 / v, qmax)
    Cs, _, _ = terms_oit(sig, 1.0)  # the centre pixel: q = 0, alpha = sigma
    Ctg = np.zeros((3, H9, W9))
    Ctg[0, 4, 4] = Cs[0]  # channel 0's residual is zero there: its sign is free
    Ct, Dt, _, Dtg = images()
    env = oracle.envelope(rec, Ct, Dt, 0.01, oracle.OIT, Ctg, Dtg, 0.0, NPX, eye_jt(), BANDS)
    assert env["n_amb"].sum() == 0
    a3 = env["allow3"][0]
    # channel 0 ranges over +-1 at that pixel: twice the unit-sign terms
    _, dLdc, dsig = terms_oit(sig, 1.0, sign=(1.0, 0.0, 0.0))
    np.testing.assert_allclose(a3[oracle.G_R], 2 * dLdc[0], rtol=1e-12)
    assert a3[oracle.G_G] == 0.0 and a3[oracle.G_B] == 0.0
    np.testing.assert_allclose(a3[oracle.G_SIG], 2 * abs(dsig), rtol=1e-12)
    # the image does not move (no counting decision is ambiguous)
    assert np.all(env["allow_C"] == 0) and env["allow_L"] == 0.0


@pytest.mark.parametrize("gap", [1e-7, 1e-5])
def test_alpha_order_of_two_gaussians_at_equal_depth(gap):
    """Two concentric Gaussians whose depths differ by `gap` of themselves: in
    the front-to-back blend, within the order band (2.3e-7 of each depth) the
    two orders are both FP32 outcomes, and at a pixel where both count they
    differ by alpha_a alpha_b (c_a - c_b) in C* (a then b: c_a a_a + c_b a_b
    (1 - a_a); b then a: c_b a_b + c_a a_a (1 - a_b); the rest, T_end C_t,
    is the same).  Outside the band, and in the order-independent blend,
    nothing is ambiguous."""
    v, d = 1.5, 0.9
    sa, sb = 0.5, 0.4
    ca, cb = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.8, 0.35])
    ra = record(4.0, 4.0, d, sa, 1 / v, 0.0, 1 / v, 2 * math.log(255 * sa), rgb=ca)
    rb = record(4.0, 4.0, d * (1 + gap), sb, 1 / v, 0.0, 1 / v, 2 * math.log(255 * sb), rgb=cb)
    rec = np.concatenate([ra, rb])
    Ct, Dt, Ctg, Dtg = images(Dt=2.0)
    ys, xs = np.mgrid[0:H9, 0:W9]
    q = ((xs - 4.0) ** 2 + (ys - 4.0) ** 2) / v
    both = q <= 2 * math.log(255 * sb)  # b's support lies inside a's
    assert np.all(np.abs(q - 2 * math.log(255 * sb)) > 1e-3)
    assert np.all(np.abs(q - 2 * math.log(255 * sa)) > 1e-3)
    env = oracle.envelope(rec, Ct, Dt, 0.01, oracle.ALPHA, Ctg, Dtg, 0.0, NPX)
    env_oit = oracle.envelope(rec, Ct, Dt, 0.01, oracle.OIT, Ctg, Dtg, 0.0, NPX)
    assert env_oit["n_amb"].sum() == 0 and np.all(env_oit["allow_C"] == 0)
    assert env["unbounded"].sum() == 0
    if gap > 2 * 2.3e-7:
        assert env["n_amb"].sum() == 0 and np.all(env["allow_C"] == 0)
        return
    np.testing.assert_array_equal(env["n_amb"] > 0, both)
    aa, ab = sa * np.exp(-0.5 * q), sb * np.exp(-0.5 * q)
    want = aa * ab * np.max(np.abs(ca - cb))
    np.testing.assert_allclose(env["allow_C"][both], want[both], rtol=1e-12)
    # D* moves by alpha_a alpha_b (d_b - d_a): a difference of two sums near
    # 1, known to their rounding
    np.testing.assert_allclose(env["allow_D"][both], (aa * ab * d * gap)[both], rtol=0, atol=1e-15)
    assert np.all(env["allow_W"] <= 1e-15)  # 1 - T_end does not depend on the order
    assert np.all(env["allow_C"][~both] == 0)


def _scene(lam=1.0):
    w = workloads.small(M=600, width=64, height=48)
    f = w.frames[0]
    vol = oracle.Volume(w.tsdf)
    oracle.fuse(vol, f.depth, f.rgb, f.cam)
    Ct, Dt, _, _ = oracle.raycast(w.tsdf, vol.sdf, vol.rgb, f.cam)
    return w, f, Ct.astype(np.float32), Dt.astype(np.float32), lam


@pytest.mark.parametrize("mode", [oracle.OIT, oracle.ALPHA])
def test_reference_gradient_is_the_adjoint_bit_for_bit(mode):
    w, f, Ct, Dt, lam = _scene()
    g64 = w.gaussians.astype(np.float64)
    ref = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                   lambda_depth=lam, mode=mode)
    JT = oracle.projection_adjoint_matrix(g64, f.cam)
    env = oracle.envelope(ref["rec"], Ct, Dt, w.eps_depth, mode, f.rgb, f.depth, lam,
                          ref["n_valid"], JT)
    np.testing.assert_array_equal(env["g2ref"], ref["g2"])
    # J^T maps the 2D gradient to the parameter gradient
    o = np.concatenate([ref["grads"][k].reshape(w.gaussians.M, -1) for k in oracle.PARAM_KEYS
                        if k in ref["grads"]], 1)
    np.testing.assert_allclose(np.einsum("mpc,mc->mp", JT, ref["g2"]), o, rtol=0,
                               atol=1e-13 * np.abs(o).max())
    assert np.all(env["s2"] >= np.abs(ref["g2"]) * (1 - 1e-12))


def test_zero_bands_give_zero_allowances():
    w, f, Ct, Dt, lam = _scene()
    g64 = w.gaussians.astype(np.float64)
    ref = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                   lambda_depth=lam)
    zero = {k: 0.0 for k in oracle.bands_for(1, 1)}
    env = oracle.envelope(ref["rec"], Ct, Dt, w.eps_depth, oracle.OIT, f.rgb, f.depth, lam,
                          ref["n_valid"], oracle.projection_adjoint_matrix(g64, f.cam), zero)
    assert env["n_amb"].sum() == 0 and env["unbounded"].sum() == 0
    assert np.all(env["allow3"] == 0) and np.all(env["allow_C"] == 0) and env["allow_L"] == 0


@pytest.mark.parametrize("mode", [oracle.OIT, oracle.ALPHA])
def test_every_flipped_combination_lies_inside_the_envelope(mode):
    """Bands 200x the FP32 ones (a few % of the pixels hold an ambiguous
    decision): the oracle re-evaluated with those decisions all inverted, or
    decided by seeded coins, moves images, loss and every parameter gradient
    by no more than the envelope."""
    w, f, Ct, Dt, lam = _scene()
    g64 = w.gaussians.astype(np.float64)
    H, W = Dt.shape
    # the order band stays at its FP32 size: the seeded flips below invert
    # counting decisions and residual signs only
    bands = {k: v * (200.0 if k not in ("res_colour", "res_depth", "order") else 1.0)
             for k, v in oracle.bands_for(W, H).items()}
    ref = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                   lambda_depth=lam, mode=mode)
    env = oracle.envelope(ref["rec"], Ct, Dt, w.eps_depth, mode, f.rgb, f.depth, lam,
                          ref["n_valid"], oracle.projection_adjoint_matrix(g64, f.cam), bands)
    assert (env["n_amb"] > 0).mean() > 0.02
    assert env["unbounded"].sum() == 0
    allow = oracle.split_params(env["allow3"], ref["grads"])
    for seed in (0, 1, 2, 3):
        alt = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                       lambda_depth=lam, mode=mode,
                                       flip=oracle.flip_spec(bands, seed))
        moved = False
        for k in ref["grads"]:
            d = np.abs(alt["grads"][k] - ref["grads"][k])
            moved = moved or d.max() > 0
            assert np.all(d <= allow[k] + 1e-12 * np.abs(ref["grads"][k]).max()), (seed, k)
        assert moved, seed
        dC = np.abs(alt["out"]["C"] - ref["out"]["C"]).max(0)
        assert np.all(dC <= env["allow_C"] + 1e-15)
        assert np.all(np.abs(alt["out"]["D"] - ref["out"]["D"]) <= env["allow_D"] + 1e-15)
        assert np.all(np.abs(alt["out"]["W"] - ref["out"]["W"]) <= env["allow_W"] + 1e-15)
        assert abs(alt["L"] - ref["L"]) <= env["allow_L"] + 1e-15


def test_too_many_ambiguous_decisions_are_flagged_unbounded():
    w, f, Ct, Dt, lam = _scene()
    g64 = w.gaussians.astype(np.float64)
    ref = oracle.render_loss_grads(g64, f.cam, Ct, Dt, f.rgb, f.depth, eps=w.eps_depth,
                                   lambda_depth=lam)
    H, W = Dt.shape
    bands = {k: v * 50.0 for k, v in oracle.bands_for(W, H).items()}
    env = oracle.envelope(ref["rec"], Ct, Dt, w.eps_depth, oracle.OIT, f.rgb, f.depth, lam,
                          ref["n_valid"], None, bands, kmax=0)
    unb = env["unbounded"] != 0
    np.testing.assert_array_equal(unb, env["n_amb"] > 0)
    assert unb.any() and np.all(np.isinf(env["allow_C"][unb]))


def test_projection_adjoint_magnitudes():
    """Magnitude arithmetic (mag.h) bounds every result of the adjoint from
    above (triangle inequality) and equals it where the chain has no sum of
    mixed signs: rgb (dL/dc passes unchanged) and the opacity logit
    (dL/dsigma sigma (1 - sigma))."""
    from datagen.scenes import with_sh
    w, f, _, _, _ = _scene()
    for gs in (w.gaussians, with_sh(w.gaussians, 2, seed=6, scale=0.05)):
        g64 = gs.astype(np.float64)
        g2 = np.random.default_rng(5).normal(size=(gs.M, oracle.G_N))
        val = oracle.project_backward(g64, f.cam, g2)
        mag = oracle.project_backward_magnitude(g64, f.cam, g2)
        assert set(mag) == set(val)
        for k in val:
            assert np.all(mag[k] >= np.abs(val[k]) * (1 - 1e-12)), k
        if gs.sh_degree == 0:
            np.testing.assert_allclose(mag["rgb"], np.abs(val["rgb"]), rtol=1e-15)
        np.testing.assert_allclose(mag["opacity_logits"], np.abs(val["opacity_logits"]), rtol=1e-14)
        # the quaternion's normalisation cancels: its magnitude exceeds |value|
        assert np.median(mag["quats"] / np.maximum(np.abs(val["quats"]), 1e-300)) > 1.0
